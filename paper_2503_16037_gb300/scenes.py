"""Seeded synthetic scenes (input data only).

This module holds no arithmetic of the radiative-transfer method: it only
synthesises the optical fields (absorption mu_a, per-species scattering
mu_s, HG asymmetry g per species) and the grid / geometry parameters that
both the CUDA library and the FP64 oracle consume.  All arrays are C-order
(z, y, x), x fastest; units are km and km^-1.

Workloads (see the design notes for the recipe):
  * ``make_plain``  -- 8x8x8 voxels of 100 m, lognormal extinction (median
    0.5 km^-1, sigma 0.5), omega 0.9, g 0.7, albedo 0.2, SZA 30, nadir view,
    26-neighbour stencil (R = 1), 8x8 pixels, FP64.
  * ``make_plume`` -- 64x64x32 voxels (50 m x 50 m x 100 m), exponential
    background aerosol plus a bent Gaussian plume of absorbing gas and plume
    aerosol; SZA 60, VZA 30, R = 2, 64x64 pixels, FP32 + FP64 refinement.
  * ``make_cloud`` -- 128x128x40 voxels of 50 m, broken cloud from a periodic
    Gaussian random field; SZA 70, VZA 20, R = 2, 128x128 pixels.
  * ``make_layered`` / ``make_random`` -- small scenes for pins and parity.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np


@dataclasses.dataclass
class Scene:
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    mu_a: np.ndarray          # (nz, ny, nx)
    mu_s: np.ndarray          # (S, nz, ny, nx)
    g: np.ndarray             # (S,)
    albedo: float
    sza: float = 30.0
    saa: float = 0.0
    vza: float = 0.0
    vaa: float = 0.0
    f0: float = 1.0
    npx: int = 8
    npy: int = 8
    R: int = 1
    M: int = 8192
    coupling: int = 1
    c_min: float = 0.0        # coupling threshold of the scattering graph (0: full stencil)
    max_couplings: int = 0    # > 0: keep this many of the largest couplings instead (c_min must be 0)
    precision: int = 0        # 0 FP64, 1 FP32 + FP64 refinement
    name: str = "scene"

    @property
    def n_species(self) -> int:
        return int(self.mu_s.shape[0])

    @property
    def n_atm(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_nodes(self) -> int:
        return self.n_atm + self.nx * self.ny

    def replace(self, **kw) -> "Scene":
        return dataclasses.replace(self, **kw)

    def copy(self) -> "Scene":
        return dataclasses.replace(self, mu_a=self.mu_a.copy(), mu_s=self.mu_s.copy(), g=self.g.copy())


def _zc(nz: int, hz: float) -> np.ndarray:
    return (np.arange(nz) + 0.5) * hz


def make_plain(seed: int = 0) -> Scene:
    """8x8x8 voxels of 100 m; extinction lognormal(ln 0.5, 0.5) km^-1."""
    nx = ny = nz = 8
    rng = np.random.Generator(np.random.PCG64(seed))
    mu_e = rng.lognormal(np.log(0.5), 0.5, (nz, ny, nx))
    omega = 0.9
    return Scene(nx, ny, nz, 0.1, 0.1, 0.1,
                 mu_a=(1.0 - omega) * mu_e, mu_s=(omega * mu_e)[None], g=np.array([0.7]),
                 albedo=0.2, sza=30.0, saa=0.0, vza=0.0, vaa=0.0, npx=8, npy=8, R=1,
                 precision=0, name="plain 8x8x8 R1")


def _plume_shape(nx, ny, nz, hx, hy, hz, sigma=0.3):
    """exp(-rho^2 / 2 sigma^2) around a bent centreline (spherical cap upwind)."""
    Lx, Ly = nx * hx, ny * hy
    x = (np.arange(nx) + 0.5) * hx
    y = (np.arange(ny) + 0.5) * hy
    z = _zc(nz, hz)
    xs, ys, zs = 0.25 * Lx, 0.5 * Ly, 0.3
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    xi = X - xs
    xip = np.maximum(xi, 0.0)
    yc = ys + 0.2 * xip ** 2 / Lx
    zc = zs + 0.3 * (1.0 - np.exp(-xip / 0.5))
    rho2 = (Y - yc) ** 2 + (Z - zc) ** 2
    rho2 = np.where(xi < 0.0, xi ** 2 + (Y - ys) ** 2 + (Z - zs) ** 2, rho2)
    return np.exp(-rho2 / (2.0 * sigma ** 2))


def make_plume(nx: int = 64, ny: int = 64, nz: int = 32, seed: int = 0, precision: int = 1,
               npx: int | None = None, npy: int | None = None, sza: float = 60.0) -> Scene:
    """Plume scene: 50 m x 50 m x 100 m voxels; species 0 background aerosol
    (0.1 km^-1 at the surface, scale height 1.5 km, omega 0.9, g 0.7),
    species 1 plume aerosol (peak 1 km^-1, omega 0.95, g 0.65); absorbing gas
    peak 2 km^-1, sigma 300 m, bent downwind.  ``seed`` is accepted for
    uniformity; the plume recipe is deterministic."""
    hx = hy = 0.05
    hz = 0.1
    z = _zc(nz, hz)
    bg = 0.1 * np.exp(-z / 1.5)[:, None, None] * np.ones((nz, ny, nx))
    shape = _plume_shape(nx, ny, nz, hx, hy, hz)
    gas = 2.0 * shape
    pa = 1.0 * shape
    mu_s = np.stack([0.9 * bg, 0.95 * pa])
    mu_a = 0.1 * bg + 0.05 * pa + gas
    return Scene(nx, ny, nz, hx, hy, hz, mu_a=mu_a, mu_s=mu_s, g=np.array([0.7, 0.65]),
                 albedo=0.1, sza=sza, saa=0.0, vza=30.0, vaa=180.0,
                 npx=npx or nx, npy=npy or ny, R=2, precision=precision,
                 name="plume %dx%dx%d R2" % (nx, ny, nz))


def periodic_grf(shape, spacing, ell: float, seed: int) -> np.ndarray:
    """Zero-mean, unit-variance periodic Gaussian random field with Gaussian
    covariance of correlation length ``ell`` (FFT filtering of white noise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal(shape)
    ks = [np.fft.fftfreq(n, d) * 2.0 * np.pi for n, d in zip(shape, spacing)]
    K = np.meshgrid(*ks, indexing="ij")
    k2 = sum(k ** 2 for k in K)
    filt = np.exp(-k2 * ell ** 2 / 4.0)
    f = np.real(np.fft.ifftn(np.fft.fftn(w) * filt))
    f -= f.mean()
    return f / f.std()


def make_cloud(nx: int = 128, ny: int = 128, nz: int = 40, seed: int = 0, precision: int = 1) -> Scene:
    """Broken cloud: 50 m voxels, G a periodic GRF (correlation 500 m);
    cloud extinction 40 max(0, G - 0.6) km^-1 between 1 and 2.5 km altitude
    (the domain top is at nz * 50 m), omega 0.999, g 0.85; clear sky
    Rayleigh-like 0.0116 exp(-z/8) km^-1, omega 1, g 0."""
    h = 0.05
    z = _zc(nz, h)
    G = periodic_grf((nz, ny, nx), (h, h, h), 0.5, seed)
    incloud = ((z >= 1.0) & (z <= 2.5))[:, None, None]
    cloud = np.where(incloud, 40.0 * np.maximum(0.0, G - 0.6), 0.0)
    ray = 0.0116 * np.exp(-z / 8.0)[:, None, None] * np.ones((nz, ny, nx))
    mu_s = np.stack([ray, 0.999 * cloud])
    mu_a = 0.001 * cloud
    return Scene(nx, ny, nz, h, h, h, mu_a=mu_a, mu_s=mu_s, g=np.array([0.0, 0.85]),
                 albedo=0.04, sza=70.0, saa=0.0, vza=20.0, vaa=0.0, npx=nx, npy=ny, R=2,
                 precision=precision, name="cloud %dx%dx%d R2" % (nx, ny, nz))


def make_layered(nx: int, ny: int, nz: int, mu_e_layers, omega_layers, g=(0.7,), albedo=0.0,
                 h=(0.1, 0.1, 0.1), R: int = 1, sza=30.0, saa=0.0, vza=0.0, vaa=0.0,
                 npx=None, npy=None, M=8192, coupling=1, precision=0) -> Scene:
    """Horizontally homogeneous layers (one species)."""
    me = np.asarray(mu_e_layers, dtype=np.float64).reshape(nz, 1, 1) * np.ones((nz, ny, nx))
    om = np.asarray(omega_layers, dtype=np.float64).reshape(-1, 1, 1)
    om = om if om.shape[0] == nz else np.full((nz, 1, 1), float(om.ravel()[0]))
    mu_s = (om * me)[None]
    mu_a = me - mu_s[0]
    return Scene(nx, ny, nz, h[0], h[1], h[2], mu_a=mu_a, mu_s=mu_s, g=np.asarray(g, dtype=np.float64),
                 albedo=albedo, sza=sza, saa=saa, vza=vza, vaa=vaa, npx=npx or nx, npy=npy or ny,
                 R=R, M=M, coupling=coupling, precision=precision, name="layered")


def make_random(nx: int, ny: int, nz: int, seed: int = 0, S: int = 2, R: int = 2,
                h=(0.05, 0.05, 0.1), sza=50.0, saa=20.0, vza=25.0, vaa=200.0, albedo=0.15,
                npx=None, npy=None, M=4096, precision=1, zero_frac: float = 0.05,
                scale: float = 1.0) -> Scene:
    """Random heterogeneous scene for parity tests: lognormal fields per
    species, a few voxels with no scattering, and random HG asymmetries."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mu_s = scale * rng.lognormal(np.log(0.4), 0.8, (S, nz, ny, nx))
    kill = rng.random((S, nz, ny, nx)) < zero_frac
    mu_s = np.where(kill, 0.0, mu_s)
    mu_a = scale * rng.lognormal(np.log(0.1), 0.8, (nz, ny, nx))
    g = rng.uniform(0.0, 0.85, S)
    return Scene(nx, ny, nz, h[0], h[1], h[2], mu_a=mu_a, mu_s=mu_s, g=g, albedo=albedo,
                 sza=sza, saa=saa, vza=vza, vaa=vaa, npx=npx or nx, npy=npy or ny, R=R, M=M,
                 precision=precision, name="random %dx%dx%d R%d" % (nx, ny, nz, R))


def workloads() -> List[str]:
    return ["plain", "plume", "cloud"]
