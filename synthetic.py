"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: only geometric test masks,
seeded random arrays and the parameter sets of the workloads (reconstruction
inputs, solver settings).  The product path and the oracle each compute
everything else on their own.

Workloads (pore spheres placed in a cube, Sec. 2 of the paper):
  small  -- 48^3 voxels at 2 nm, d ~ Normal(20, 5) nm clipped to [6, 40],
            overlap tolerance 0.5, porosity 0.40; tau = 1, g = 1e-6,
            maximal-inscribed-sphere pore size, T = 300 K, methane.
  sweep  -- 256^3 at 1 nm, d ~ Normal(30, 8) nm, overlap tolerance 0.3,
            porosity in {0.15, 0.25, 0.35, 0.45}; 13-direction pore size.
  batch  -- 150 structures, edge in {64, 96, 128, 160, 200}, porosity
            U[0.10, 0.50], <d> U[10, 60] nm with sd = <d>/4, tolerance
            U[0, 0.8], 1.5 nm voxels (the paper's resolution).
  large  -- 512^3, porosity 0.30, d ~ Normal(40, 10) nm, tolerance 0.5.
"""
from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class Recon:
    seed: int
    shape: tuple
    dx_nm: float
    mean_nm: float
    sd_nm: float
    dmin_nm: float
    dmax_nm: float
    porosity: float
    xi: float
    p0: float = 0.5
    dist: int = 0  # 0 Normal clipped, 1 Uniform(mean - sd, mean + sd)
    max_trials: int = 20_000_000

    def with_(self, **kw):
        return replace(self, **kw)


def small_structure(seed=1):
    return Recon(seed, (48, 48, 48), 2.0, 20.0, 5.0, 6.0, 40.0, 0.40, 0.5)


def sweep_structure(porosity, seed=1, edge=256):
    return Recon(seed, (edge, edge, edge), 1.0, 30.0, 8.0, 6.0, 54.0, porosity, 0.3)


SWEEP_POROSITIES = (0.15, 0.25, 0.35, 0.45)


def large_structure(seed=1, edge=512):
    return Recon(seed, (edge, edge, edge), 1.0, 40.0, 10.0, 10.0, 70.0, 0.30, 0.5)


def batch_structures(n=150, seed=7):
    """The 150-structure set: per structure (edge, porosity, <d>, tolerance)
    drawn from a seeded generator; voxel 1.5 nm; clipped at <d> +- 3 sd."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        edge = int(rng.choice([64, 96, 128, 160, 200]))
        eps = float(rng.uniform(0.10, 0.50))
        mean = float(rng.uniform(10.0, 60.0))
        xi = float(rng.uniform(0.0, 0.8))
        sd = 0.25 * mean
        out.append(Recon(1000 + i, (edge, edge, edge), 1.5, mean, sd, max(3.0, mean - 3 * sd),
                         mean + 3 * sd, eps, xi))
    return out


def campaign_structures(means=(30.0, 45.0, 60.0), porosities=None, xis=(0.1, 0.2, 0.3), seeds=5, edge=200,
                        dx_nm=1.5):
    """The paper's reconstruction campaign (Sec. 2): pore diameters uniform in
    <d> +- 15 nm, <d> in {30, 45, 60} nm, porosity 0.10 .. 0.55 in steps of
    0.05, overlap tolerance in {0.1, 0.2, 0.3}, five structures per
    configuration, 200^3 voxels of 1.5 nm.  Any sub-grid (and a smaller box
    for tests) can be asked for."""
    porosities = porosities if porosities is not None else tuple(round(0.10 + 0.05 * k, 2) for k in range(10))
    out = []
    for i, (mean, eps, xi) in enumerate((m, e, x) for m in means for e in porosities for x in xis):
        for s in range(seeds):
            out.append(Recon(100_000 + 100 * i + s, (edge, edge, edge), dx_nm, mean, 15.0, mean - 15.0,
                             mean + 15.0, eps, xi, dist=1))
    return out


# ------------------------------------------------------------------ geometric masks
def slit(nx, H, nz=1):
    """Two plane walls normal to y: pore rows y = 1..H, solid rows y = 0, H+1."""
    m = np.zeros((nx, H + 2, nz), np.uint8)
    m[:, 1:H + 1, :] = 1
    return m


def layered_slit(nx, H, nz=1):
    """slit() plus an integer layer index per pore row (1..H), for layered
    pore sizes."""
    m = slit(nx, H, nz)
    layer = np.zeros(m.shape, np.int32)
    for y in range(1, H + 1):
        layer[:, y, :] = y
    return m, layer


def square_duct(nx, a):
    """Square duct of side a (pore) along x with a one-voxel solid frame."""
    m = np.zeros((nx, a + 2, a + 2), np.uint8)
    m[:, 1:a + 1, 1:a + 1] = 1
    return m


def tube(nx, R, n=None):
    """Circular tube of radius R voxels along x; pore where the voxel centre
    lies within R of the axis."""
    n = n or (2 * int(np.ceil(R)) + 2)
    c = n / 2.0
    y = np.arange(n) + 0.5
    Y, Z = np.meshgrid(y, y, indexing="ij")
    disk = ((Y - c) ** 2 + (Z - c) ** 2) <= R * R
    return np.broadcast_to(disk, (nx, n, n)).astype(np.uint8).copy()


def sphere_in_cube(L):
    """Cube of side L with a solid sphere of diameter L at its centre; the
    pore space is the rest (porosity -> 1 - pi/6)."""
    x = np.arange(L) + 0.5
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    c = L / 2.0
    solid = ((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2) <= (L / 2.0) ** 2
    return (~solid).astype(np.uint8)


def bcc_array(L, porosity):
    """Cube of side L holding one cell of a body-centred cubic array of equal
    solid spheres (at the corners, with their periodic images, and at the
    centre), their diameter set by the porosity of the continuous array,
    1 - 2 (pi/6) d^3 / L^3; the pore space is the rest."""
    d = L * ((1.0 - porosity) * 6.0 / (2.0 * np.pi)) ** (1.0 / 3.0)
    x = np.arange(L) + 0.5
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    solid = np.zeros((L, L, L), bool)
    for cx, cy, cz in [(a, b, c) for a in (0.0, L) for b in (0.0, L) for c in (0.0, L)] + [(L / 2.0,) * 3]:
        solid |= ((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) <= (d / 2.0) ** 2
    return (~solid).astype(np.uint8), d


def offset_channel(nx=12, ny=10, nz=3, shift=4):
    """Two half-length slits along x, rows y = 1, 2 for x < nx/2 and rows
    y = 1+shift, 2+shift for x >= nx/2, joined by a riser at x = nx/2 - 1,
    nx/2.  The structure spans x, but with shift >= 3 no D3Q19 link joins
    the x = nx-1 face to the x = 0 face across the periodic boundary; with
    shift = 2 one diagonal link per z layer does."""
    m = np.zeros((nx, ny, nz), np.uint8)
    h = nx // 2
    m[:h, 1:3, :] = 1
    m[h:, 1 + shift:3 + shift, :] = 1
    m[h - 1:h + 1, 1:3 + shift, :] = 1
    return m


def closed_box(shape):
    """Pore interior with a one-voxel solid shell on every face."""
    m = np.zeros(shape, np.uint8)
    m[1:-1, 1:-1, 1:-1] = 1
    return m


def random_mask(shape, p, seed):
    """Bernoulli(p) pore voxels."""
    return (np.random.default_rng(seed).random(shape) < p).astype(np.uint8)


def blob_mask(shape, seed, n=6, rmin=1.5, rmax=4.0):
    """Union of a few random balls (periodic in y, z) -- a tiny stand-in for a
    reconstructed structure, used where a test needs pores of several sizes."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    m = np.zeros(shape, bool)
    X, Y, Z = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5, np.arange(nz) + 0.5, indexing="ij")
    for _ in range(n):
        c = rng.random(3) * np.array(shape)
        r = rng.uniform(rmin, rmax)
        dy = np.abs(Y - c[1]); dy = np.minimum(dy, ny - dy)
        dz = np.abs(Z - c[2]); dz = np.minimum(dz, nz - dz)
        m |= (X - c[0]) ** 2 + dy ** 2 + dz ** 2 <= r * r
    # a channel along x so that something percolates
    y0, z0 = rng.integers(0, ny), rng.integers(0, nz)
    m[:, y0, z0] = True
    return m.astype(np.uint8)


def random_field(shape, seed, lo=-1.0, hi=1.0, dtype=np.float64):
    return np.random.default_rng(seed).uniform(lo, hi, size=shape).astype(dtype)
