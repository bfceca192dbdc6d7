"""Seeded synthetic inputs for the staggered-channel pressure-Poisson workloads.

This module is shared by the CPU oracle (``oracle/``), the GPU tests and ``bench.py``.
It only *draws* inputs: grid faces, random velocity fields, weight fields and the
manufactured right-hand side sampled at cell centres.  It contains none of the
solver's arithmetic (no divergence, gradient, transform or tridiagonal solve).

Conventions (the channel of Sec. 2, Fig. 1-2, with the axis naming of Sec. 5:
x streamwise and periodic, y wall-normal and bounded, z spanwise and periodic):

* real cell fields are C-ordered ``(Ny, Nz, Nx)`` (x fastest);
* ``u[j, k, i]`` sits on the x-face at ``x = i*dx`` (left face of cell i);
* ``w[j, k, i]`` sits on the z-face at ``z = k*dz``;
* ``v[j, k, i]`` for ``j = 0..Ny`` sits on the y-face ``y_faces[j]``; ``v[0]`` and
  ``v[Ny]`` are the two walls;
* pressure sits at cell centres ``((i+1/2)dx, (y_j+y_{j+1})/2, (k+1/2)dz)``.

Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64), drawn in C order,
components in the order u, v, w.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

LX = 2.0 * math.pi
LZ = math.pi


@dataclass(frozen=True)
class ChannelCase:
    """A named channel workload: grid sizes, domain and tanh stretching factor."""
    name: str
    nx: int
    ny: int
    nz: int
    stretch: float
    lx: float = LX
    lz: float = LZ

    @property
    def npoints(self) -> int:
        return self.nx * self.ny * self.nz


# The workloads of the method's precision / batching forms, named by what they are.
CHANNEL_32 = ChannelCase("channel_32x32x32_tanh1.5", 32, 32, 32, 1.5)
CHANNEL_512 = ChannelCase("channel_512x384x512_tanh2.0", 512, 384, 512, 2.0)
CHANNEL_1536 = ChannelCase("channel_1536x768x1024_tanh2.2", 1536, 768, 1024, 2.2)
CHANNEL_256 = ChannelCase("channel_256x192x256_tanh1.8", 256, 192, 256, 1.8)


def tanh_faces(ny: int, stretch: float) -> np.ndarray:
    """Wall-normal face coordinates y_j = tanh(s(2j/Ny - 1)) / tanh(s), j = 0..Ny, on [-1, 1]."""
    j = np.arange(ny + 1, dtype=np.float64)
    y = np.tanh(stretch * (2.0 * j / ny - 1.0)) / np.tanh(stretch)
    y[0], y[-1] = -1.0, 1.0
    return y


def uniform_faces(ny: int) -> np.ndarray:
    """Uniform wall-normal faces on [-1, 1]."""
    y = np.linspace(-1.0, 1.0, ny + 1)
    y[0], y[-1] = -1.0, 1.0
    return y


def random_velocity(seed: int, nx: int, ny: int, nz: int, scale: float = 1.0,
                    walls_zero: bool = False):
    """Seeded N(0, scale^2) staggered velocity (u, v, w); optionally zero v on both walls."""
    rng = np.random.default_rng(seed)
    u = scale * rng.standard_normal((ny, nz, nx))
    v = scale * rng.standard_normal((ny + 1, nz, nx))
    w = scale * rng.standard_normal((ny, nz, nx))
    if walls_zero:
        v[0] = 0.0
        v[-1] = 0.0
    return u, v, w


def poiseuille_plus_noise(seed: int, case: ChannelCase, noise: float = 0.1):
    """Laminar profile u = 1 - y^2 at u-points plus seeded N(0, noise^2) on every component.

    The no-penetration walls keep v = 0 on both wall faces.
    """
    faces = tanh_faces(case.ny, case.stretch)
    yc = 0.5 * (faces[:-1] + faces[1:])
    u, v, w = random_velocity(seed, case.nx, case.ny, case.nz, scale=noise, walls_zero=True)
    u += (1.0 - yc * yc)[:, None, None]
    return u, v, w


def weight_field(seed: int, nx: int, ny: int, nz: int):
    """Seeded U(-1, 1) weights for each velocity component (loss sum(w . u))."""
    rng = np.random.default_rng(seed)
    wu = rng.uniform(-1.0, 1.0, (ny, nz, nx))
    wv = rng.uniform(-1.0, 1.0, (ny + 1, nz, nx))
    ww = rng.uniform(-1.0, 1.0, (ny, nz, nx))
    return wu, wv, ww


def random_field(seed: int, shape) -> np.ndarray:
    """Seeded N(0, 1) array of the given shape."""
    return np.random.default_rng(seed).standard_normal(shape)


def manufactured_rhs(nx: int, ny: int, nz: int, faces: np.ndarray,
                     lx: float = LX, lz: float = LZ) -> np.ndarray:
    """cos(2 pi x / Lx) cos(4 pi z / Lz) cos(pi y / 2) sampled at the pressure points."""
    x = (np.arange(nx) + 0.5) * (lx / nx)
    z = (np.arange(nz) + 0.5) * (lz / nz)
    yc = 0.5 * (faces[:-1] + faces[1:])
    return (np.cos(np.pi * yc / 2.0)[:, None, None]
            * np.cos(4.0 * np.pi * z / lz)[None, :, None]
            * np.cos(2.0 * np.pi * x / lx)[None, None, :])



BATCH_NX_NZ = (64, 96, 128, 192, 256, 384)
BATCH_NY = (48, 64, 96, 128, 192)


def batch_instances(seed: int = 5, count: int = 64):
    """Uneven-size batch: per instance, in order, Nx and Nz from BATCH_NX_NZ, Ny from BATCH_NY and
    the tanh stretching from U(1.0, 2.5), all drawn from one default_rng(seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx = int(rng.choice(BATCH_NX_NZ))
        nz = int(rng.choice(BATCH_NX_NZ))
        ny = int(rng.choice(BATCH_NY))
        s = float(rng.uniform(1.0, 2.5))
        out.append(ChannelCase(f"batch_{nx}x{ny}x{nz}_tanh{s:.3f}", nx, ny, nz, s))
    return out
