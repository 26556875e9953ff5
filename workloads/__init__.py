"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and bench.py.

This module builds problem descriptions only: label volumes, optical-property tables,
sources, detectors and run settings.  It holds none of the photon-transport arithmetic
(no hop sampling, no Fresnel, no scattering, no deposition), so both sides of every
parity test can take their inputs from here without sharing any of the method.

The workloads are the paper's benchmarks B1/B2/B2a (60x60x60 mm^3 cube, pencil beam at
(30,30,0) along +z, optional r=15 mm sphere; the benchmark description beside Fig. 2)
and five synthetic configurations of the same kind:

  c1  64^3, 1 mm voxels, homogeneous (mua 0.01, mus 10, g 0.9, n 1.37) in air,
      pencil beam (32,32,0) +z, 1e5 photons, one 0-5 ns gate
  c2  c1 plus two spherical inclusions, 10 gates of 0.5 ns, 4 disk detectors, 1e8 photons
  c3  256x256x128, 0.5 mm voxels, 4 planar layers, Gaussian beam of 2 mm waist,
      50 gates of 0.1 ns, 1e9 photons
  c4  256 seeded random volumes (side 32..128, 1-3 ellipsoids), 5 gates of 1 ns

Conventions (shared input layout, not method arithmetic):
  * labels: uint8 array indexed [z, y, x] (x fastest in memory); label 0 is the exterior.
  * media: float64 array [n_media, 4] = (mua /mm, mus /mm, g, n); row 0 is the exterior
    and only its n is used.
  * a voxel takes an inclusion's label when the voxel centre lies inside (<= r^2);
    inclusions are painted in the listed order, so later ones overwrite earlier ones.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

C0_MM_PER_NS = 299.792458  # speed of light in vacuum, mm/ns


@dataclasses.dataclass
class Workload:
    name: str
    labels: np.ndarray                  # uint8 [nz, ny, nx]
    voxel_mm: float
    media: np.ndarray                   # float64 [n_media, 4]
    src_kind: int                       # 0 pencil, 1 gaussian
    src_pos: Tuple[float, float, float]
    src_dir: Tuple[float, float, float]
    waist_mm: float
    detectors: np.ndarray               # float64 [n_det, 4] = cx, cy, cz, r (mm)
    n_photons: int
    n_gates: int
    dt_ns: float
    reflect: int = 1
    seed: int = 12345
    max_detected: int = 0

    @property
    def shape(self) -> Tuple[int, int, int]:
        nz, ny, nx = self.labels.shape
        return nx, ny, nz

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def _grid_centres(nx: int, ny: int, nz: int, h: float):
    z = (np.arange(nz) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    x = (np.arange(nx) + 0.5) * h
    return np.meshgrid(z, y, x, indexing="ij")


def paint_sphere(labels: np.ndarray, h: float, centre, radius: float, label: int) -> None:
    """Paint `label` into every voxel whose centre lies within the sphere."""
    nz, ny, nx = labels.shape
    zc, yc, xc = _grid_centres(nx, ny, nz, h)
    cx, cy, cz = centre
    inside = (xc - cx) ** 2 + (yc - cy) ** 2 + (zc - cz) ** 2 <= radius * radius
    labels[inside] = label


def paint_ellipsoid(labels: np.ndarray, h: float, centre, semi_axes, label: int) -> None:
    """Paint `label` into every voxel whose centre lies within the axis-aligned ellipsoid."""
    nz, ny, nx = labels.shape
    zc, yc, xc = _grid_centres(nx, ny, nz, h)
    cx, cy, cz = centre
    ax, ay, az = semi_axes
    inside = ((xc - cx) / ax) ** 2 + ((yc - cy) / ay) ** 2 + ((zc - cz) / az) ** 2 <= 1.0
    labels[inside] = label


def paint_layers(labels: np.ndarray, h: float, thickness_mm: List[float]) -> None:
    """Planar layers along +z from z=0: label k+1 for the k-th thickness, the last label
    filling the remainder of the volume."""
    nz = labels.shape[0]
    z0 = 0
    lab = 1
    for th in thickness_mm:
        nvox = int(round(th / h))
        labels[z0:min(nz, z0 + nvox)] = lab
        z0 += nvox
        lab += 1
    labels[min(nz, z0):] = lab


AIR = (0.0, 0.0, 1.0, 1.0)
TISSUE_C1 = (0.01, 10.0, 0.9, 1.37)


def c1(n_photons: int = 100_000, seed: int = 12345) -> Workload:
    """64^3 homogeneous scattering cube in air, pencil beam, one 0-5 ns gate."""
    labels = np.ones((64, 64, 64), dtype=np.uint8)
    media = np.array([AIR, TISSUE_C1], dtype=np.float64)
    return Workload("c1_homogeneous_64", labels, 1.0, media, 0, (32.0, 32.0, 0.0),
                    (0.0, 0.0, 1.0), 0.0, np.zeros((0, 4)), n_photons, 1, 5.0, 1, seed)


C2_DETECTORS = np.array([[22.0, 32.0, 0.0, 2.0],
                         [42.0, 32.0, 0.0, 2.0],
                         [32.0, 22.0, 0.0, 2.0],
                         [32.0, 42.0, 0.0, 2.0]], dtype=np.float64)


def c2(n_photons: int = 100_000_000, seed: int = 12345) -> Workload:
    """64^3 background with two overlapping spheres (the second painted last), 10 gates
    of 0.5 ns, four r=2 mm disk detectors on the z=0 face 10 mm from the source."""
    labels = np.ones((64, 64, 64), dtype=np.uint8)
    paint_sphere(labels, 1.0, (32.0, 32.0, 24.0), 10.0, 2)
    paint_sphere(labels, 1.0, (20.0, 40.0, 30.0), 8.0, 3)
    media = np.array([AIR, TISSUE_C1, (0.05, 5.0, 0.9, 1.37), (0.002, 1.0, 0.8, 1.45)],
                     dtype=np.float64)
    return Workload("c2_two_spheres_64", labels, 1.0, media, 0, (32.0, 32.0, 0.0),
                    (0.0, 0.0, 1.0), 0.0, C2_DETECTORS.copy(), n_photons, 10, 0.5, 1, seed,
                    max_detected=10_000_000)


def c3(n_photons: int = 1_000_000_000, seed: int = 12345) -> Workload:
    """256x256x128 volume of 0.5 mm voxels, layers 3/7/2/rest mm, Gaussian beam of
    2 mm waist at the top-face centre, 50 gates of 0.1 ns."""
    labels = np.zeros((128, 256, 256), dtype=np.uint8)
    paint_layers(labels, 0.5, [3.0, 7.0, 2.0])
    media = np.array([AIR,
                      (0.019, 7.8, 0.89, 1.37),
                      (0.019, 9.4, 0.89, 1.37),
                      (0.004, 0.01, 0.89, 1.37),
                      (0.02, 6.6, 0.89, 1.37)], dtype=np.float64)
    return Workload("c3_layers_256x256x128", labels, 0.5, media, 1, (64.0, 64.0, 0.0),
                    (0.0, 0.0, 1.0), 2.0, np.zeros((0, 4)), n_photons, 50, 0.1, 1, seed)


def c4(n_sims: int = 256, seed: int = 1711032440) -> List[Workload]:
    """Seeded batch of uneven simulations: cubic volumes of side {32,48,64,96,128} mm,
    1-3 random axis-aligned ellipsoids, random optical properties, log-uniform photon
    counts in [1e5, 1e7], pencil source at a random point of the z=0 face, 5 gates of 1 ns."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_sims):
        side = int(rng.choice([32, 48, 64, 96, 128]))
        n_inc = int(rng.integers(1, 4))
        labels = np.ones((side, side, side), dtype=np.uint8)
        rows = [AIR]
        for _ in range(n_inc + 1):
            mua = float(10 ** rng.uniform(-3, -1))
            mus = float(rng.uniform(0.5, 20.0))
            g = float(rng.uniform(0.5, 0.95))
            n = float(rng.uniform(1.33, 1.45))
            rows.append((mua, mus, g, n))
        for i in range(n_inc):
            centre = rng.uniform(0.2 * side, 0.8 * side, size=3)
            semi = rng.uniform(0.1 * side, 0.3 * side, size=3)
            paint_ellipsoid(labels, 1.0, tuple(centre), tuple(semi), i + 2)
        sx, sy = rng.uniform(0.0, side, size=2)
        n_ph = int(round(10 ** rng.uniform(5, 7)))
        out.append(Workload(f"c4_sim{k:03d}_side{side}", labels, 1.0,
                            np.array(rows, dtype=np.float64), 0, (float(sx), float(sy), 0.0),
                            (0.0, 0.0, 1.0), 0.0, np.zeros((0, 4)), n_ph, 5, 1.0, 1,
                            seed + 1 + k))
    return out


def c5(n_volumes: int, seed: int, n_photons: int = 100_000) -> List[Workload]:
    """Seeded 64 mm cubes for the learned denoiser, drawn like c4 with the side fixed at
    64: 1-3 random axis-aligned ellipsoids, random optical properties, pencil source at a
    random point of the z=0 face, one 0-5 ns gate.  Different generator seeds give
    different volumes (training and held-out sets); the simulation seed of volume k is
    seed + 1 + k, so consecutive generator seeds share photon streams between different
    volumes, which differ in geometry and optics (the trajectories do not coincide)."""
    rng = np.random.default_rng(seed)
    side = 64
    out = []
    for k in range(n_volumes):
        n_inc = int(rng.integers(1, 4))
        labels = np.ones((side, side, side), dtype=np.uint8)
        rows = [AIR]
        for _ in range(n_inc + 1):
            rows.append((float(10 ** rng.uniform(-3, -1)), float(rng.uniform(0.5, 20.0)),
                         float(rng.uniform(0.5, 0.95)), float(rng.uniform(1.33, 1.45))))
        for i in range(n_inc):
            centre = rng.uniform(0.2 * side, 0.8 * side, size=3)
            semi = rng.uniform(0.1 * side, 0.3 * side, size=3)
            paint_ellipsoid(labels, 1.0, tuple(centre), tuple(semi), i + 2)
        sx, sy = rng.uniform(0.0, side, size=2)
        out.append(Workload(f"c5_vol{k:04d}", labels, 1.0, np.array(rows, dtype=np.float64), 0,
                            (float(sx), float(sy), 0.0), (0.0, 0.0, 1.0), 0.0, np.zeros((0, 4)),
                            n_photons, 1, 5.0, 1, seed + 1 + k))
    return out


def paper_b(variant: str = "B1", n_photons: int = 100_000_000, seed: int = 12345) -> Workload:
    """The paper's benchmarks: 60 mm cube (mua 0.005, mus 1.0, g 0.01, n 1.37) in air,
    pencil beam at (30,30,0) +z.  B2/B2a add a central r=15 mm sphere (mua 0.002, mus 5.0,
    g 0.9, n 1.0).  B1 terminates photons at the cube boundary (no reflection); B2/B2a
    apply Fresnel/Snell at the sphere and cube boundaries.  (B2 and B2a differ only in
    non-atomic vs atomic accumulation; the library always accumulates race-free.)
    The paper states no time window; one 0-5 ns gate is used here (reading)."""
    labels = np.ones((60, 60, 60), dtype=np.uint8)
    media = [AIR, (0.005, 1.0, 0.01, 1.37)]
    if variant.upper() in ("B2", "B2A"):
        paint_sphere(labels, 1.0, (30.0, 30.0, 30.0), 15.0, 2)
        media.append((0.002, 5.0, 0.9, 1.0))
    reflect = 0 if variant.upper() == "B1" else 1
    return Workload(f"paper_{variant.lower()}_60", labels, 1.0, np.array(media), 0,
                    (30.0, 30.0, 0.0), (0.0, 0.0, 1.0), 0.0, np.zeros((0, 4)), n_photons, 1,
                    5.0, reflect, seed)


def by_name(name: str, **kw) -> Workload:
    table = {"c1": c1, "c2": c2, "c3": c3}
    if name in table:
        return table[name](**kw)
    if name.lower() in ("b1", "b2", "b2a"):
        return paper_b(name.upper(), **kw)
    raise KeyError(name)
