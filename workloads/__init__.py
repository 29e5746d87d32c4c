"""Seeded synthetic inputs for the finite-frequency traveltime tomography path.

This module is shared by the FP64 oracle and by the CUDA path, so it holds none of
the method's arithmetic: no sensitivity kernel, no spectrum integral, no operator.
It only builds the inputs the method is applied to:

* transducer rings and the emitter-receiver pair list (Sec. II-C, Eq. forward_compact:
  one row of F per emitter-receiver pair; unordered pairs s < r since the kernel is
  reciprocal in s and r),
* the voxel grid (Sec. III: a regular grid of voxel centres, midpoint rule),
* velocity perturbation phantoms, traveltime noise, PSF spike positions and ring
  subsets.

Every random draw comes from ``numpy.random.default_rng(seed)`` with the seed fixed
per workload, so both sides see bit-identical inputs.

Units are SI throughout: metres, seconds, m/s.

The five workloads mirror the configurations the project is measured on:

1. ``ring32``: 32 transducers on a 50 mm ring, 496 pairs, 48x48x16 voxels at 2 mm,
   5 Gaussian blobs, 10 CG iterations.
2. ``ring256``: 256 transducers on a 100 mm ring, 32640 pairs, 200x200x40 voxels at
   1 mm (1.6 M voxels), three nested cylinders, 30 CG iterations.
3. ``ring32_diff``: the ``ring32`` sizes, used for gradient / precision studies.
4. ``slices3d``: the 256-element ring stepped to 16 z positions 4 mm apart (pairs only
   within a slice, 522240 per band), three frequency bands, 256x256x96 voxels at
   0.75 mm, 12 random ellipsoidal inclusions, 20 CG iterations.
5. ``psf3d``: the ``slices3d`` geometry with 128 seeded spikes and ring subsets of
   64 / 128 / 256 elements.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Water sound speed used by the synthetic workloads (m/s).
C0_WATER = 1500.0
# Standard deviation of the Gaussian traveltime noise (s).
NOISE_SIGMA_S = 5e-9


@dataclasses.dataclass(frozen=True)
class Grid:
    """Regular voxel grid. Voxel (i, j, k) has its centre at origin + (i, j, k) * h.

    The linear voxel index is v = (k * ny + j) * nx + i (x fastest).
    """

    nx: int
    ny: int
    nz: int
    h: float
    origin: Tuple[float, float, float]

    @property
    def n_vox(self) -> int:
        return self.nx * self.ny * self.nz

    @staticmethod
    def centred(nx: int, ny: int, nz: int, h: float) -> "Grid":
        """Grid whose voxel centres sit at (i - (n-1)/2) * h about the ring centre."""
        return Grid(nx, ny, nz, h, (-(nx - 1) * h / 2, -(ny - 1) * h / 2, -(nz - 1) * h / 2))

    def centres(self) -> np.ndarray:
        """(V, 3) float64 array of voxel centres in linear-index order."""
        i = np.arange(self.nx)
        j = np.arange(self.ny)
        k = np.arange(self.nz)
        kk, jj, ii = np.meshgrid(k, j, i, indexing="ij")
        x = self.origin[0] + ii.ravel() * self.h
        y = self.origin[1] + jj.ravel() * self.h
        z = self.origin[2] + kk.ravel() * self.h
        return np.stack([x, y, z], axis=1)

    def axis(self, a: int) -> np.ndarray:
        n = (self.nx, self.ny, self.nz)[a]
        return self.origin[a] + np.arange(n) * self.h


@dataclasses.dataclass(frozen=True)
class Band:
    """Gaussian power spectrum W(omega) of one frequency band (centre and std in Hz)."""

    f_center_hz: float
    f_sigma_hz: float
    n_samples: int = 4096
    periods: float = 3.0

    @property
    def dt_max(self) -> float:
        """Cut-off detour time: `periods` dominant periods of the band."""
        return self.periods / self.f_center_hz


@dataclasses.dataclass
class Workload:
    name: str
    tx: np.ndarray            # (n_tx, 3) float64 transducer positions
    pairs: np.ndarray         # (P, 2) int32 (s, r) with s < r, row order
    band_of_row: np.ndarray   # (M,) int32 band index per row; rows = bands x pairs
    bands: List[Band]
    grid: Grid
    c0: float
    cg_iters: int
    lambda_rel: float
    model_seed: Optional[int] = None
    noise_seed: Optional[int] = None

    @property
    def n_rows(self) -> int:
        return int(self.band_of_row.shape[0])

    def row_pairs(self) -> np.ndarray:
        """(M, 2) int32 emitter/receiver indices of every row (bands repeat the pairs)."""
        return np.tile(self.pairs, (len(self.bands), 1))


def ring(n_tx: int, radius: float, z: float = 0.0) -> np.ndarray:
    """Transducers evenly on a ring: x_k = (rho cos 2 pi k/n, rho sin 2 pi k/n, z)."""
    ang = 2.0 * np.pi * np.arange(n_tx) / n_tx
    return np.stack([radius * np.cos(ang), radius * np.sin(ang), np.full(n_tx, z)], axis=1)


def unordered_pairs(idx: Sequence[int]) -> np.ndarray:
    """All unordered pairs (s, r), s < r, in lexicographic order of (s, r)."""
    idx = list(idx)
    out = [(idx[a], idx[b]) for a in range(len(idx)) for b in range(a + 1, len(idx))]
    return np.asarray(out, dtype=np.int32).reshape(-1, 2)


def slice_rings(n_tx: int, radius: float, z_positions: Sequence[float]) -> Tuple[np.ndarray, np.ndarray]:
    """One ring per z position; pairs only within a slice, ordered (slice, s, r)."""
    tx = np.concatenate([ring(n_tx, radius, z) for z in z_positions], axis=0)
    pairs = np.concatenate(
        [unordered_pairs(range(s * n_tx, (s + 1) * n_tx)) for s in range(len(z_positions))], axis=0
    )
    return tx, pairs


def roi_pixels(radius: float, h: float, half_offset: bool = False) -> np.ndarray:
    """In-plane pixel centres of a 2-D inversion grid over a circular region of interest
    (Sec. IV's lab inversion: 1 mm pixels over a 70 mm-radius ROI): the points (i h, j h) with
    x^2 + y^2 <= radius^2, or ((i + 1/2) h, (j + 1/2) h) with ``half_offset``. Returned as an
    (n, 2) array, x fastest. The test is exact in integers when radius / h is an integer."""
    q = radius / h
    n = int(math.floor(q)) + 1
    k = np.arange(-n, n + 1, dtype=np.int64)
    if half_offset:
        a = 2 * k + 1                     # 2 (k + 1/2): twice the coordinate in pixels
        ax, ay = np.meshgrid(a, a)
        if abs(q - round(q)) < 1e-9:
            inside = ax * ax + ay * ay <= 4 * round(q) ** 2
        else:
            inside = (ax * ax + ay * ay) <= (2.0 * q) ** 2
        xy = np.stack([ax[inside], ay[inside]], axis=1) * (0.5 * h)
    else:
        ix, iy = np.meshgrid(k, k)
        if abs(q - round(q)) < 1e-9:
            inside = ix * ix + iy * iy <= round(q) ** 2
        else:
            inside = (ix * ix + iy * iy) <= q * q
        xy = np.stack([ix[inside], iy[inside]], axis=1) * h
    return xy.astype(np.float64)


def lab_ascan_count(n_emitters: int = 16, n_receivers: int = 16, n_positions: int = 11,
                    n_rotations: int = 23) -> int:
    """A-scans of Sec. IV's lab acquisition: two 16-element arrays (every emitter of one to
    every receiver of the other), 11 receiver-array positions and 23 rotations of the
    set-up. One traveltime, i.e. one row of the forward operator, per A-scan."""
    return n_emitters * n_receivers * n_positions * n_rotations


# --------------------------------------------------------------------------- phantoms

def blobs_model(grid: Grid, seed: int, n_blobs: int = 5, amp: float = 30.0,
                sigma_range=(3e-3, 8e-3), disc_radius: float = 35e-3,
                z_range=(-8e-3, 8e-3)) -> np.ndarray:
    """Sum of Gaussian blobs: sigma ~ U[3, 8] mm, amplitude +-amp with a random sign,
    centres uniform in a disc of radius 35 mm and z ~ U[-8, 8] mm. float64 (V,)."""
    rng = np.random.default_rng(seed)
    sig = rng.uniform(*sigma_range, size=n_blobs)
    sign = rng.choice([-1.0, 1.0], size=n_blobs)
    rad = disc_radius * np.sqrt(rng.uniform(0.0, 1.0, size=n_blobs))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n_blobs)
    zc = rng.uniform(*z_range, size=n_blobs)
    ctr = np.stack([rad * np.cos(phi), rad * np.sin(phi), zc], axis=1)
    x = grid.centres()
    m = np.zeros(x.shape[0])
    for b in range(n_blobs):
        d2 = np.sum((x - ctr[b]) ** 2, axis=1)
        m += sign[b] * amp * np.exp(-0.5 * d2 / sig[b] ** 2)
    return m


def cylinders_model(grid: Grid, radii=(20e-3, 40e-3, 60e-3), values=(40.0, -25.0, 15.0)) -> np.ndarray:
    """Nested concentric cylinders along z, innermost wins. float64 (V,)."""
    x = grid.centres()
    rho = np.hypot(x[:, 0], x[:, 1])
    m = np.zeros(x.shape[0])
    for r, v in sorted(zip(radii, values), reverse=True):
        m[rho < r] = v
    return m


def ellipsoids_model(grid: Grid, seed: int, count: int = 12, amp: float = 40.0,
                     semi_range=(4e-3, 15e-3), disc_radius: float = 70e-3,
                     z_half: float = 30e-3) -> np.ndarray:
    """Random ellipsoidal inclusions with random orientation, +-amp m/s, later ones on top."""
    rng = np.random.default_rng(seed)
    x = grid.centres()
    m = np.zeros(x.shape[0])
    for _ in range(count):
        semi = rng.uniform(*semi_range, size=3)
        q, _r = np.linalg.qr(rng.normal(size=(3, 3)))
        rad = disc_radius * np.sqrt(rng.uniform())
        phi = rng.uniform(0, 2 * np.pi)
        c = np.array([rad * np.cos(phi), rad * np.sin(phi), rng.uniform(-z_half, z_half)])
        val = amp * rng.choice([-1.0, 1.0])
        loc = (x - c) @ q
        inside = np.sum((loc / semi) ** 2, axis=1) <= 1.0
        m[inside] = val
    return m


def noise(n_rows: int, seed: int, sigma: float = NOISE_SIGMA_S) -> np.ndarray:
    """Gaussian traveltime noise N(0, sigma^2), float64 (M,)."""
    return np.random.default_rng(seed).normal(0.0, sigma, size=n_rows)


def random_voxels(grid: Grid, n: int, seed: int, rho_max: float = 70e-3, z_max: float = 30e-3) -> np.ndarray:
    """Seeded distinct voxel indices uniformly over voxels with rho <= rho_max, |z| <= z_max."""
    x = grid.centres()
    ok = np.flatnonzero((np.hypot(x[:, 0], x[:, 1]) <= rho_max) & (np.abs(x[:, 2]) <= z_max))
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(ok, size=n, replace=False)).astype(np.int64)


# --------------------------------------------------------------------------- workloads

def ring32() -> Workload:
    """32 transducers, 50 mm ring, 496 pairs, 48x48x16 voxels at 2 mm (36864 voxels)."""
    tx = ring(32, 50e-3)
    pairs = unordered_pairs(range(32))
    bands = [Band(1.0e6, 0.3e6)]
    return Workload("ring32", tx, pairs, np.zeros(len(pairs), np.int32), bands,
                    Grid.centred(48, 48, 16, 2e-3), C0_WATER, cg_iters=10, lambda_rel=1e-3,
                    model_seed=1, noise_seed=2)


def ring256() -> Workload:
    """256 transducers, 100 mm ring, 32640 pairs, 200x200x40 voxels at 1 mm (1.6 M voxels)."""
    tx = ring(256, 100e-3)
    pairs = unordered_pairs(range(256))
    bands = [Band(1.0e6, 0.4e6)]
    return Workload("ring256", tx, pairs, np.zeros(len(pairs), np.int32), bands,
                    Grid.centred(200, 200, 40, 1e-3), C0_WATER, cg_iters=30, lambda_rel=1e-3,
                    model_seed=None, noise_seed=3)


def slices3d() -> Workload:
    """16 rings of 256 at z = -30..30 mm step 4 mm, 522240 pairs x 3 bands, 256x256x96 at 0.75 mm."""
    zpos = [-30e-3 + 4e-3 * s for s in range(16)]
    tx, pairs = slice_rings(256, 100e-3, zpos)
    bands = [Band(0.6e6, 0.2e6), Band(1.0e6, 0.2e6), Band(1.4e6, 0.2e6)]
    bor = np.repeat(np.arange(3, dtype=np.int32), len(pairs))
    return Workload("slices3d", tx, pairs, bor, bands, Grid.centred(256, 256, 96, 0.75e-3),
                    C0_WATER, cg_iters=20, lambda_rel=1e-3, model_seed=6, noise_seed=7)


def elevation_stack(spacing: float, n_positions: int, n_tx: int = 256) -> Workload:
    """One 100 mm ring of n_tx elements translated to n_positions elevations spaced by `spacing`
    (centred on z = 0), pairs within each elevation, one band (1 MHz, sigma 0.4 MHz), on a
    141 x 141 x 33 grid at 1 mm (a cylinder-sized ROI of radius 70 mm and height 32 mm, with
    voxel centres on the axes). Used for the 3 mm vs 8 mm elevation-spacing comparison."""
    zpos = [spacing * (k - (n_positions - 1) / 2.0) for k in range(n_positions)]
    tx, pairs = slice_rings(n_tx, 100e-3, zpos)
    return Workload(f"stack{int(round(spacing * 1e4))}", tx, pairs, np.zeros(len(pairs), np.int32),
                    [Band(1.0e6, 0.4e6)], Grid.centred(141, 141, 33, 1e-3), C0_WATER, cg_iters=20,
                    lambda_rel=1e-3)


def ring_subsets(n_tx: int = 256, n_slices: int = 16, strides=(4, 2, 1), n_bands: int = 3) -> List[np.ndarray]:
    """Row subsets of a (band, slice, s, r) pair list: every 4th / 2nd / every element of each ring.

    A pair belongs to a subset when both its elements are on the subset's stride. Returned
    as sorted row-index arrays, for all bands (3 for ``slices3d``, 1 for ``ring256``).
    """
    ppr = n_tx * (n_tx - 1) // 2
    local = unordered_pairs(range(n_tx))
    out = []
    for st in strides:
        keep = np.flatnonzero((local[:, 0] % st == 0) & (local[:, 1] % st == 0))
        rows = [b * n_slices * ppr + s * ppr + keep for b in range(n_bands) for s in range(n_slices)]
        out.append(np.concatenate(rows).astype(np.int32))
    return out


def gaussian_block(n: int, b: int, seed: int) -> np.ndarray:
    """(n, b) float64 standard normal test block (a randomized eigensolver's starting matrix),
    columns stored contiguously when transposed: block.T is (b, n) C-ordered."""
    return np.random.default_rng(seed).standard_normal((b, n)).T


def model_for(w: Workload) -> np.ndarray:
    """The velocity perturbation (m/s, float64) that goes with a workload."""
    if w.name.startswith("ring32"):
        return blobs_model(w.grid, w.model_seed)
    if w.name.startswith("ring256"):
        return cylinders_model(w.grid)
    if w.name == "slices3d":
        return ellipsoids_model(w.grid, w.model_seed)
    if w.name == "slices32":
        return ellipsoids_model(w.grid, w.model_seed, semi_range=(3e-3, 8e-3), disc_radius=35e-3, z_half=12e-3)
    raise KeyError(w.name)


def ring256_3band() -> Workload:
    """ring256's array and grid with the three bands of slices3d (0.6 / 1.0 / 1.4 MHz, sigma
    0.2 MHz; the 1.4 MHz band does not vanish at its cut-off): 97920 rows, 1.6 M voxels."""
    base = ring256()
    bands = [Band(0.6e6, 0.2e6), Band(1.0e6, 0.2e6), Band(1.4e6, 0.2e6)]
    bor = np.repeat(np.arange(3, dtype=np.int32), len(base.pairs))
    return Workload("ring256_3band", base.tx, base.pairs, bor, bands, base.grid, base.c0, cg_iters=base.cg_iters,
                    lambda_rel=base.lambda_rel, model_seed=base.model_seed, noise_seed=base.noise_seed)


def slices32() -> Workload:
    """A small slice-by-slice acquisition of the slices3d kind: the 32-element 50 mm ring stepped
    to 4 z positions 4 mm apart (pairs only within a slice), the three bands of slices3d
    (0.6 / 1.0 / 1.4 MHz, sigma 0.2 MHz), 48 x 48 x 24 voxels at 2 mm, random ellipsoidal
    inclusions, 20 CG iterations: 3 x 4 x 496 = 5952 rows, 55296 voxels."""
    zpos = [-6e-3 + 4e-3 * s for s in range(4)]
    tx, pairs = slice_rings(32, 50e-3, zpos)
    bands = [Band(0.6e6, 0.2e6), Band(1.0e6, 0.2e6), Band(1.4e6, 0.2e6)]
    bor = np.repeat(np.arange(3, dtype=np.int32), len(pairs))
    return Workload("slices32", tx, pairs, bor, bands, Grid.centred(48, 48, 24, 2e-3), C0_WATER,
                    cg_iters=20, lambda_rel=1e-3, model_seed=6, noise_seed=7)


def by_name(name: str) -> Workload:
    return {"ring32": ring32, "ring256": ring256, "slices3d": slices3d, "ring256_3band": ring256_3band,
            "slices32": slices32}[name]()


def tiny(n_tx: int = 12, radius: float = 20e-3, n: Tuple[int, int, int] = (14, 14, 6),
         h: float = 2e-3, f_center: float = 1.0e6, f_sigma: float = 0.3e6, z: float = 0.0) -> Workload:
    """Small ring for dense-matrix checks (few thousand voxels, tens of pairs)."""
    tx = ring(n_tx, radius, z)
    pairs = unordered_pairs(range(n_tx))
    return Workload("tiny", tx, pairs, np.zeros(len(pairs), np.int32), [Band(f_center, f_sigma)],
                    Grid.centred(*n, h), C0_WATER, cg_iters=10, lambda_rel=1e-3)
