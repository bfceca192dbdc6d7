"""Grid metrics of the staggered channel (Sec. 2, Fig. 2) and the eigenvalues of Eq. 9.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Grid:
    """Uniform x and z, stretched y given by its Ny+1 face coordinates.

    0-based wall-normal indexing: cell j lies between faces y[j] and y[j+1];
    ``dy[j] = y[j+1] - y[j]``; ``yc[j]`` is the cell centre; for an interior face
    j = 1..Ny-1, ``h[j] = yc[j] - yc[j-1]`` is the centre-to-centre distance across it.
    """
    nx: int
    nz: int
    faces: np.ndarray
    lx: float = 2.0 * math.pi
    lz: float = math.pi
    ny: int = field(init=False)

    def __post_init__(self):
        self.faces = np.asarray(self.faces, dtype=np.float64)
        self.ny = self.faces.size - 1
        self.dx = self.lx / self.nx
        self.dz = self.lz / self.nz
        self.dy = np.diff(self.faces)
        self.yc = 0.5 * (self.faces[:-1] + self.faces[1:])
        h = np.full(self.ny + 1, np.nan)
        h[1:self.ny] = self.yc[1:] - self.yc[:-1]
        self.h = h

    # --- the wall-normal three-point operator, row j (0-based) ------------------
    # (L_y p)_j = [ (p_{j+1}-p_j)/h_{j+1} - (p_j-p_{j-1})/h_j ] / dy_j, with the
    # wall fluxes (faces 0 and Ny) set to zero (homogeneous Neumann).
    @property
    def lower(self) -> np.ndarray:
        """a_j: coefficient of p_{j-1} in row j (0 for the bottom row)."""
        a = np.zeros(self.ny)
        a[1:] = 1.0 / (self.dy[1:] * self.h[1:self.ny])
        return a

    @property
    def upper(self) -> np.ndarray:
        """c_j: coefficient of p_{j+1} in row j (0 for the top row)."""
        c = np.zeros(self.ny)
        c[:-1] = 1.0 / (self.dy[:-1] * self.h[1:self.ny])
        return c

    # --- modified wavenumbers (eigenvalues of the periodic 3-point stencils) ----
    def lambda_x(self) -> np.ndarray:
        """lambda_x(kx) = -(4/dx^2) sin^2(pi kx / Nx), kx = 0..Nx-1 (Eq. 9)."""
        kx = np.arange(self.nx)
        return -(4.0 / self.dx ** 2) * np.sin(np.pi * kx / self.nx) ** 2

    def lambda_z(self) -> np.ndarray:
        """lambda_z(kz) = -(4/dz^2) sin^2(pi kz / Nz), kz = 0..Nz-1 (Eq. 9)."""
        kz = np.arange(self.nz)
        return -(4.0 / self.dz ** 2) * np.sin(np.pi * kz / self.nz) ** 2

    @property
    def volume_weights(self) -> np.ndarray:
        """Per-row weights dy_j used for the compatibility condition and the gauge."""
        return self.dy
