"""Seeded synthetic inputs for the DDA hot path.

This module is shared by the CPU oracle, the CUDA binding's tests and the
benchmark.  It holds target geometry, incident directions, polarization
vectors and random test vectors -- the *inputs* of the method -- and none of
its arithmetic (no polarizabilities, no interaction matrix, no solver, no
cross sections).

Target grids follow the user guide's conventions (section "Target
Generation", ELLIPSOID and RCTGLPRSM shapes): a rectangular computational
volume nx*ny*nz, one composition code per lattice site (0 = vacuum,
1..ncomp = material), stored with x fastest, i.e. ``grid[iz, iy, ix]``.
Dipole centres sit at half-integer offsets about the box centre,
``r = (ix-(nx-1)/2, iy-(ny-1)/2, iz-(nz-1)/2)`` in lattice units.

The five named workloads are the synthetic stand-ins for the guide's
example targets (ELLIPSOID, RCTGLPRSM; the guide's ``examples_exp`` files
are not available): a 16^3 sphere, a 64^3 sphere, a 3:2:1 ellipsoid on a
96x64x32 lattice with 64 seeded directions x 2 polarizations, a 48x48x24
two-material block with a seeded Bernoulli composition, and a 256^3 sphere
with 8 seeded directions x 2 polarizations.  Two more: ``aubrick32x64x64``,
the guide's FROM_FILE sample (a full 32x64x64 Au block), and
``spheroid64x64x256``, a small target with the 256^3 sphere's 512-point z
transform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_DIRECTIONS = 20120214
SEED_COMPOSITION = 20120514


def ellipsoid_grid(nx: int, ny: int, nz: int, dx: float, dy: float, dz: float) -> np.ndarray:
    """ELLIPSOID target: site occupied iff (x/dx)^2+(y/dy)^2+(z/dz)^2 <= 1/4.

    dx, dy, dz are the full axis lengths in lattice units (ELLIPSOID
    section: SHPAR_i are the lengths along x, y, z).  Returns uint8 [nz,ny,nx].
    """
    x = (np.arange(nx) - (nx - 1) / 2.0) / dx
    y = (np.arange(ny) - (ny - 1) / 2.0) / dy
    z = (np.arange(nz) - (nz - 1) / 2.0) / dz
    inside = (z[:, None, None] ** 2 + y[None, :, None] ** 2 + x[None, None, :] ** 2) <= 0.25
    return inside.astype(np.uint8)


def sphere_grid(n: int, diameter: float | None = None) -> np.ndarray:
    """Pseudosphere in an n^3 box; diameter defaults to n (|r| <= n/2)."""
    d = float(n if diameter is None else diameter)
    return ellipsoid_grid(n, n, n, d, d, d)


def block_bernoulli_grid(nx: int, ny: int, nz: int, p: float = 0.5,
                         seed: int = SEED_COMPOSITION) -> np.ndarray:
    """Fully occupied RCTGLPRSM block; each site is composition 1 with
    probability p, else composition 2 (numpy PCG64 stream from ``seed``)."""
    rng = np.random.default_rng(seed)
    u = rng.random((nz, ny, nx))
    return np.where(u < p, 1, 2).astype(np.uint8)


def uniform_directions(n: int, seed: int = SEED_DIRECTIONS) -> np.ndarray:
    """n unit vectors uniform on the sphere: z ~ U(-1,1), phi ~ U(0, 2pi)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def polarization_pair(khat: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Two real orthonormal polarizations transverse to each direction:
    e1 = normalize(z x k) (x-hat when k is along z), e2 = k x e1."""
    khat = np.atleast_2d(np.asarray(khat, dtype=np.float64))
    zc = np.cross(np.array([0.0, 0.0, 1.0]), khat)
    nrm = np.linalg.norm(zc, axis=1)
    e1 = np.where(nrm[:, None] < 1e-8, np.array([1.0, 0.0, 0.0]), zc / np.maximum(nrm, 1e-300)[:, None])
    e2 = np.cross(khat, e1)
    return e1, e2


def random_complex(shape, seed: int) -> np.ndarray:
    """Seeded complex128 array with standard-normal real and imaginary parts."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@dataclass
class Workload:
    """One synthetic scattering problem: grid, materials, size parameter, RHS."""
    name: str
    grid: np.ndarray                 # uint8 [nz, ny, nx]
    m: list                          # complex refractive index per composition
    x: float                         # size parameter 2*pi*a_eff/lambda
    khat: np.ndarray                 # (R, 3) real unit propagation directions
    ehat: np.ndarray                 # (R, 3) complex polarization vectors
    mode: str                        # "fp64", "fp32_refined"
    tol: float = 1e-5
    notes: dict = field(default_factory=dict)

    @property
    def shape(self):
        nz, ny, nx = self.grid.shape
        return nx, ny, nz

    @property
    def ndipoles(self) -> int:
        return int(np.count_nonzero(self.grid))

    @property
    def nrhs(self) -> int:
        return int(self.khat.shape[0])


def _k_along_x_two_pols():
    khat = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    ehat = np.array([[0, 1, 0], [0, 0, 1]], dtype=np.complex128)
    return khat, ehat


def _sweep(ndir: int, seed: int = SEED_DIRECTIONS):
    k = uniform_directions(ndir, seed)
    e1, e2 = polarization_pair(k)
    khat = np.repeat(k, 2, axis=0)
    ehat = np.empty((2 * ndir, 3), dtype=np.complex128)
    ehat[0::2] = e1
    ehat[1::2] = e2
    return khat, ehat


def workload(name: str) -> Workload:
    """The named synthetic workloads (see module docstring)."""
    if name == "sphere16":
        k, e = _k_along_x_two_pols()
        return Workload(name, sphere_grid(16), [1.33 + 0.01j], 1.0, k, e, "fp64")
    if name == "sphere64":
        k, e = _k_along_x_two_pols()
        return Workload(name, sphere_grid(64), [1.5 + 0.02j], 5.0, k, e, "fp32_refined")
    if name == "ellipsoid96x64x32":
        k, e = _sweep(64)
        return Workload(name, ellipsoid_grid(96, 64, 32, 96, 64, 32), [1.33 + 0.05j], 8.0, k, e,
                        "fp32_refined")
    if name == "block48x48x24":
        khat = np.array([[1.0, 0.0, 0.0]])
        ehat = np.array([[0, 1, 0]], dtype=np.complex128)
        return Workload(name, block_bernoulli_grid(48, 48, 24), [1.7 + 0.3j, 1.2 + 0.01j], 4.0,
                        khat, ehat, "fp64")
    if name == "sphere256":
        k, e = _sweep(8)
        return Workload(name, sphere_grid(256), [1.33 + 0.01j], 20.0, k, e, "fp32_refined")
    if name == "aubrick32x64x64":
        # the guide's FROM_FILE sample: a 0.5 x 1 x 1 micron Au block as a
        # 32 x 64 x 64 array, m = 0.9656 + 1.8628i, lambda = 0.5 micron,
        # aeff = 0.49237 micron (x = 2 pi aeff / lambda), k along the short axis
        k, e = _k_along_x_two_pols()
        return Workload(name, np.ones((64, 64, 32), np.uint8), [0.9656 + 1.8628j], 2 * np.pi * 0.49237 / 0.5, k, e,
                        "fp32_refined")
    if name == "spheroid64x64x256":
        # profiler-capture stand-in for sphere256: its 128x128x512 padded grid
        # has the same 512-point z transform at 1/16 of the memory
        k, e = _sweep(8)
        return Workload(name, ellipsoid_grid(64, 64, 256, 64, 64, 256), [1.33 + 0.01j], 10.0, k, e,
                        "fp32_refined")
    raise KeyError(name)


WORKLOADS = ("sphere16", "sphere64", "ellipsoid96x64x32", "block48x48x24", "sphere256")
