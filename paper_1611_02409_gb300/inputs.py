"""Seeded synthetic initial fields (rho, u, T), in the paper's dimensionless units.

This module holds no arithmetic of the scheme: it only draws the macroscopic fields
that both the CUDA path and the oracle start from.  Every generator returns float64
numpy arrays in the library's field layout: rho[ny, nx], u[D, ny, nx], T[ny, nx] (3-D:
[nz, ny, nx]).  Noise is uniform in (-a, a) from numpy's PCG64 with the given seed,
drawn in the order rho, u_x, u_y, (u_z), T.
"""
from __future__ import annotations

import numpy as np


def _noise(rng, shape, amp):
    return rng.uniform(-amp, amp, size=shape) if amp else np.zeros(shape)


def shear_thermal_wave(nx=64, ny=64, u_amp=0.01, T_amp=0.001, noise=1e-6, seed=0):
    """rho = 1, u_x = u_amp sin(2 pi y/ny), u_y = 0, T = 1 + T_amp sin(2 pi x/nx), plus noise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    rho = 1.0 + _noise(rng, (ny, nx), noise)
    u = np.stack([u_amp * np.sin(2 * np.pi * y / ny) + _noise(rng, (ny, nx), noise),
                  _noise(rng, (ny, nx), noise)])
    T = 1.0 + T_amp * np.sin(2 * np.pi * x / nx) + _noise(rng, (ny, nx), noise)
    return rho, u, T


def taylor_green_2d(n=4096, U0=0.02, T_amp=0.01, noise=0.0, seed=0, ny=None):
    """Thermal Taylor-Green field, k = 2 pi / n:
    u = U0 (sin kx cos ky, -cos kx sin ky), T = 1 + T_amp cos kx cos ky, rho = 1."""
    nx, ny = n, ny or n
    rng = np.random.Generator(np.random.PCG64(seed))
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    x = np.arange(nx, dtype=float)[None, :]
    y = np.arange(ny, dtype=float)[:, None]
    sx, cx, sy, cy = np.sin(kx * x), np.cos(kx * x), np.sin(ky * y), np.cos(ky * y)
    rho = 1.0 + _noise(rng, (ny, nx), noise)
    u = np.stack([U0 * sx * cy + _noise(rng, (ny, nx), noise), -U0 * cx * sy + _noise(rng, (ny, nx), noise)])
    T = 1.0 + T_amp * cx * cy + _noise(rng, (ny, nx), noise)
    return rho, u, T


def taylor_green_3d(n=256, U0=0.02, T_amp=0.01, noise=1e-6, seed=0):
    """3-D thermal Taylor-Green vortex, k = 2 pi / n:
    u = U0 (sin x cos y cos z, -cos x sin y cos z, 0), T = 1 + T_amp cos x cos y cos z."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = 2 * np.pi / n
    z, y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), np.arange(n, dtype=float),
                          indexing="ij")
    s = (n, n, n)
    rho = 1.0 + _noise(rng, s, noise)
    u = np.stack([U0 * np.sin(k * x) * np.cos(k * y) * np.cos(k * z) + _noise(rng, s, noise),
                  -U0 * np.cos(k * x) * np.sin(k * y) * np.cos(k * z) + _noise(rng, s, noise),
                  _noise(rng, s, noise)])
    T = 1.0 + T_amp * np.cos(k * x) * np.cos(k * y) * np.cos(k * z) + _noise(rng, s, noise)
    return rho, u, T


def random_fields(shape, seed=0, drho=0.02, du=0.03, dT=0.03):
    """Smooth-free random fields for element-wise parity: rho = 1 + U(-drho, drho), etc."""
    rng = np.random.Generator(np.random.PCG64(seed))
    D = len(shape)
    rho = 1.0 + rng.uniform(-drho, drho, size=shape)
    u = rng.uniform(-du, du, size=(D,) + tuple(shape))
    T = 1.0 + rng.uniform(-dT, dT, size=shape)
    return rho, u, T


def rest_channel(nx=4, ny=256):
    """rho = 1, u = 0, T = 1 on an nx x ny channel (thermal Couette start)."""
    return np.ones((ny, nx)), np.zeros((2, ny, nx)), np.ones((ny, nx))


def shear_wave(n=64, nx=4, amp=1e-3):
    """rho = T = 1, u_x = amp sin(2 pi y/n), u_y = 0 on an nx x n periodic strip."""
    y = np.arange(n, dtype=float)[:, None] * np.ones((1, nx))
    return np.ones((n, nx)), np.stack([amp * np.sin(2 * np.pi * y / n), np.zeros((n, nx))]), np.ones((n, nx))


def isobaric_thermal_wave(n=64, ny=4, amp=1e-3):
    """T = 1 + amp sin(2 pi x/n), rho = 1/T (uniform pressure), u = 0 on an n x ny strip."""
    x = np.arange(n, dtype=float)[None, :] * np.ones((ny, 1))
    T = 1.0 + amp * np.sin(2 * np.pi * x / n)
    return 1.0 / T, np.zeros((2, ny, n)), T
