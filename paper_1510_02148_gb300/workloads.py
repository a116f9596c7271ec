"""Seeded synthetic inputs: permeability fields, sources, boundary conditions,
subdomain grids and levelset thresholds.

This module holds none of the solver's arithmetic; both the CUDA path and the
CPU oracle consume what it produces.  The fields imitate the layered and
heterogeneous reservoirs of the paper's experiments (Section 2, the layered
"sandwich" field behind Theorem 3.1; Section 4, the layered BO/SPE5/SAGD
cases and the SPE10-sized model).  No dataset is read or reproduced: every
field is generated from a seed.

Array convention: fields are numpy arrays shaped (nz, ny, nx), x fastest, so
cell (ix, iy, iz) has flat index (iz * ny + iy) * nx + ix.
Boundary faces are ordered -x, +x, -y, +y, -z, +z; type 0 = no-flow,
1 = Dirichlet (the cells of that face hold the given value).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

NOFLOW, DIRICHLET = 0, 1
X_DIRICHLET = ((DIRICHLET, DIRICHLET, NOFLOW, NOFLOW, NOFLOW, NOFLOW), (1.0, 0.0, 0.0, 0.0, 0.0, 0.0))


@dataclasses.dataclass
class Problem:
    """One pressure system: K, q, boundary conditions and the SLD setup."""
    name: str
    K: np.ndarray                  # (nz, ny, nx) float64 permeability
    q: Optional[np.ndarray]        # (nz, ny, nx) float64 source, or None
    bc_type: Tuple[int, ...]
    bc_value: Tuple[float, ...]
    S: Tuple[int, int, int]        # subdomains (Sx, Sy, Sz)
    tau: Tuple[float, ...]         # L-1 ascending levelset thresholds
    L: int
    tol: float = 1e-9

    @property
    def shape(self):
        return self.K.shape

    @property
    def n(self):
        return int(self.K.size)

    @property
    def d(self):
        return int(self.S[0] * self.S[1] * self.S[2] * self.L)


def layered(nx, ny, nz, n_layers, high=1.0, low=1e-6, bottom_high=True) -> np.ndarray:
    """Horizontal layers stacked in z, alternating high/low; layer of cell iz is
    floor(iz * n_layers / nz); layer 0 (bottom) is the high value."""
    iz = np.arange(nz)
    layer = (iz * n_layers) // nz
    is_high = (layer % 2 == 0) if bottom_high else (layer % 2 == 1)
    col = np.where(is_high, high, low).astype(np.float64)
    return np.broadcast_to(col[:, None, None], (nz, ny, nx)).copy()


def lognormal_layered(nx, ny, nz, n_layers, med_high=1.0, med_low=1e-4, sigma=1.0,
                      seed=1) -> np.ndarray:
    """Layered medians (alternating med_high / med_low, bottom high) times an
    i.i.d. lognormal factor exp(sigma * xi), xi ~ N(0, 1) per cell."""
    base = layered(nx, ny, nz, n_layers, med_high, med_low)
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal(base.shape)
    return base * np.exp(sigma * xi)


def _random_rotation(rng) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def inclusions(nx, ny, nz, frac=0.20, k_background=1.0, k_inclusion=1e-6, a_range=(16, 96),
               seed=1, max_count=100000) -> Tuple[np.ndarray, float]:
    """Background K with randomly placed, randomly rotated ellipsoids of
    k_inclusion: 'lens' (a, a, a/8) or 'channel' (a, a/6, a/6), a ~ U[a_range],
    added until the marked fraction reaches `frac`.  Returns (K, fraction)."""
    rng = np.random.default_rng(seed)
    mask = np.zeros((nz, ny, nx), dtype=bool)
    n = mask.size
    marked = 0
    a_lo, a_hi = a_range
    for _ in range(max_count):
        if marked >= frac * n:
            break
        c = rng.uniform([0, 0, 0], [nx, ny, nz])
        a = rng.uniform(a_lo, a_hi)
        semi = np.array([a, a, a / 8.0]) if rng.random() < 0.5 else np.array([a, a / 6.0, a / 6.0])
        R = _random_rotation(rng)
        r = int(math.ceil(semi.max()))
        x0, x1 = max(0, int(c[0]) - r), min(nx, int(c[0]) + r + 1)
        y0, y1 = max(0, int(c[1]) - r), min(ny, int(c[1]) + r + 1)
        z0, z1 = max(0, int(c[2]) - r), min(nz, int(c[2]) + r + 1)
        if x0 >= x1 or y0 >= y1 or z0 >= z1:
            continue
        zz, yy, xx = np.meshgrid(np.arange(z0, z1) + 0.5 - c[2], np.arange(y0, y1) + 0.5 - c[1],
                                 np.arange(x0, x1) + 0.5 - c[0], indexing="ij")
        # body coordinates u = R^T (p - c)
        u0 = R[0, 0] * xx + R[1, 0] * yy + R[2, 0] * zz
        u1 = R[0, 1] * xx + R[1, 1] * yy + R[2, 1] * zz
        u2 = R[0, 2] * xx + R[1, 2] * yy + R[2, 2] * zz
        inside = (u0 / semi[0]) ** 2 + (u1 / semi[1]) ** 2 + (u2 / semi[2]) ** 2 <= 1.0
        sub = mask[z0:z1, y0:y1, x0:x1]
        marked += int(np.count_nonzero(inside & ~sub))
        sub |= inside
    K = np.where(mask, k_inclusion, k_background).astype(np.float64)
    return K, marked / n


def point_source(nx, ny, nz, value=1.0, at=None) -> np.ndarray:
    q = np.zeros((nz, ny, nx))
    ix, iy, iz = at if at is not None else (nx // 2, ny // 2, nz // 2)
    q[iz, iy, ix] = value
    return q


# ---------------------------------------------------------------------------
# The five workloads.  Sizes are parameters so tests can build smaller copies
# with the same structure.
# ---------------------------------------------------------------------------
def layered_sandwich(nx=32, ny=32, nz=32, n_layers=8, S=(2, 2, 2), low=1e-6) -> Problem:
    """32^3, 8 z-layers of 4 cells alternating 1.0 / 1e-6, Dirichlet p=1 at
    x=0 and p=0 at x=nx-1, q=0, 2x2x2 subdomains x 2 levelsets = 16 vectors."""
    K = layered(nx, ny, nz, n_layers, 1.0, low)
    return Problem(f"layered{nx}x{ny}x{nz}", K, None, *X_DIRICHLET, S=S,
                   tau=(math.sqrt(low),), L=2)


def lognormal_point_source(nx=256, ny=256, nz=128, n_layers=16, S=(4, 4, 4), seed=1) -> Problem:
    """256x256x128, 16 z-layers of lognormal(sigma=1) K with medians 1 / 1e-4,
    Dirichlet x-faces, q=+1 at the centre cell, 4x4x4 subdomains x 2 levelsets."""
    K = lognormal_layered(nx, ny, nz, n_layers, 1.0, 1e-4, 1.0, seed)
    return Problem(f"lognormal{nx}x{ny}x{nz}", K, point_source(nx, ny, nz), *X_DIRICHLET,
                   S=S, tau=(1e-2,), L=2)


def inclusion_field(nx=512, ny=512, nz=256, S=(8, 8, 8), frac=0.20, seed=1,
                    a_range=(16, 96)) -> Tuple[Problem, float]:
    """512x512x256 background K=1 with tilted lens/channel inclusions at 1e-6
    covering >= 20% of the volume, Dirichlet x-faces, 8x8x8 subdomains x 3
    levelsets = 1536 vectors (thresholds 1e-4, 1e-2: the middle class stays
    empty for this binary field)."""
    K, f = inclusions(nx, ny, nz, frac, 1.0, 1e-6, a_range, seed)
    return Problem(f"inclusions{nx}x{ny}x{nz}", K, None, *X_DIRICHLET, S=S,
                   tau=(1e-4, 1e-2), L=3), f


def batch(count=64, side_range=(32, 160), seed=1) -> List[Problem]:
    """`count` cubes, side ~ U{32..160}, layered K with contrast 1e4 and
    layer count ~ U{4..16}, S^3 subdomains with S ~ U{2,3,4}, 2 levelsets."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        side = int(rng.integers(side_range[0], side_range[1] + 1))
        layers = int(rng.integers(4, 17))
        S = int(rng.integers(2, 5))
        K = layered(side, side, side, layers, 1.0, 1e-4)
        out.append(Problem(f"batch{j}_{side}", K, None, *X_DIRICHLET, S=(S, S, S),
                           tau=(1e-2,), L=2))
    return out


def learned_field(seed, n=128, contrast_range=(4.0, 6.0), S=(4, 4, 2)) -> Problem:
    """128^3 lognormal-layered field with contrast 10^c, c ~ U[4, 6], layer
    count ~ U{4..16}; 4x4x2 subdomains x 2 levelsets = 64 SLD vectors."""
    rng = np.random.default_rng(10_000_019 + seed)
    c = float(rng.uniform(*contrast_range))
    layers = int(rng.integers(4, 17))
    K = lognormal_layered(n, n, n, layers, 1.0, 10.0 ** (-c), 1.0, seed)
    return Problem(f"learned{seed}", K, None, *X_DIRICHLET, S=S, tau=(10.0 ** (-c / 2),), L=2)


def sandwich_theorem(nx=4, ny=4, nz=12, n_layers=6, eps=1e-6) -> Problem:
    """Tiny layered field for the eigenvalue count of Theorem 3.1: no-flow on
    all faces except Dirichlet (p=0) on the top (+z) face."""
    K = layered(nx, ny, nz, n_layers, 1.0, eps)
    bct = (NOFLOW, NOFLOW, NOFLOW, NOFLOW, NOFLOW, DIRICHLET)
    return Problem(f"theorem{nx}x{ny}x{nz}", K, None, bct, (0, 0, 0, 0, 0, 0.0),
                   S=(1, 1, n_layers), tau=(math.sqrt(eps),), L=2)


def _smooth2(a, passes=3, w=5):
    """Separable box smoothing in the last two axes (x and y), `passes` times."""
    k = np.ones(w) / w
    for _ in range(passes):
        a = np.apply_along_axis(lambda v: np.convolve(v, k, mode="same"), -1, a)
        a = np.apply_along_axis(lambda v: np.convolve(v, k, mode="same"), -2, a)
    return a


def spe10_like(nx=180, ny=220, nz=85, S=(2, 2, 2), seed=1) -> Problem:
    """An SPE10-shaped synthetic field (the SPE10 data are not used): the top
    35/85 of the layers a smooth, strongly varying lognormal field (log10 K
    spread ~ 4 decades, like the Tarbert formation), the rest fluvial: sinuous
    high-permeability channels (~1e3) a few cells wide and a few layers thick
    in a low-permeability background (~1e-2), like the Upper Ness; clipped to
    [1e-3, 10^4.5], about SPE10's 7.5 decades.  Dirichlet
    x-faces, a unit source at the centre cell, plain subdomain deflation
    (L = 1: one vector per subdomain, d = Sx * Sy * Sz), as in the paper's
    SPE10 runs with d = 8, 27, 64."""
    rng = np.random.default_rng(seed)
    ntop = int(round(nz * 35 / 85))
    K = np.empty((nz, ny, nx))
    g = _smooth2(rng.standard_normal((nz, ny, nx)), passes=2, w=5)
    g = (g - g.mean()) / g.std()
    # top: lognormal, log10 K ~ N(1, 1.2^2)
    K[nz - ntop:] = 10.0 ** (1.0 + 1.2 * g[nz - ntop:])
    # bottom: background, then channels
    nb = nz - ntop
    K[:nb] = 10.0 ** (-2.0 + 0.3 * g[:nb])
    y = np.arange(ny)
    xg = np.arange(nx)[None, :]
    z = 0
    while z < nb:
        thick = int(rng.integers(2, 6))
        for _ in range(int(rng.integers(2, 6))):
            x0 = rng.uniform(0, nx)
            amp = rng.uniform(0.05, 0.2) * nx
            lam = rng.uniform(0.3, 1.0) * ny
            ph = rng.uniform(0, 2 * np.pi)
            width = rng.uniform(2.0, 0.06 * nx + 3.0)
            xc = x0 + amp * np.sin(2 * np.pi * y / lam + ph)
            inside = np.abs(xg - xc[:, None]) < width / 2
            for dz in range(thick):
                if z + dz < nb:
                    K[z + dz][inside] = 10.0 ** (3.0 + 0.3 * g[z + dz][inside])
        z += thick + int(rng.integers(0, 3))
    # SPE10's permeabilities span about 7.5 decades
    K = np.clip(K, 1e-3, 10.0 ** 4.5)
    return Problem(f"spe10like{nx}x{ny}x{nz}", K, point_source(nx, ny, nz), *X_DIRICHLET, S=S, tau=(), L=1)
