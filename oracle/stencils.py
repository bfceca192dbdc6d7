"""Staggered second-order finite-volume operators (Sec. 2, Fig. 2, Eqs. 4, 7, 8).

Test infrastructure only (see the package docstring).

Field layouts (C order, x fastest): cell fields ``(Ny, Nz, Nx)``; ``u`` and ``w`` face
fields ``(Ny, Nz, Nx)`` with ``u[j,k,i]`` on the face between cells i-1 and i (periodic);
``v`` ``(Ny+1, Nz, Nx)`` with ``v[j]`` on face ``y[j]`` (``v[0]``, ``v[Ny]`` are walls).
"""
from __future__ import annotations

import numpy as np

from .grid import Grid


def divergence(g: Grid, u, v, w):
    """(D u)_{jki} = (u_{i+1}-u_i)/dx + (v_{j+1}-v_j)/dy_j + (w_{k+1}-w_k)/dz."""
    du = (np.roll(u, -1, axis=2) - u) / g.dx
    dw = (np.roll(w, -1, axis=1) - w) / g.dz
    dv = (v[1:] - v[:-1]) / g.dy[:, None, None]
    return du + dv + dw


def gradient(g: Grid, p):
    """G p on the faces: x and z periodic differences; y interior faces only (walls 0)."""
    gx = (p - np.roll(p, 1, axis=2)) / g.dx
    gz = (p - np.roll(p, 1, axis=1)) / g.dz
    gy = np.zeros((g.ny + 1,) + p.shape[1:])
    gy[1:g.ny] = (p[1:] - p[:-1]) / g.h[1:g.ny, None, None]
    return gx, gy, gz


def laplacian(g: Grid, p):
    """L_h p = D G p written out: 3-point stencils in x, z and the stretched y (Eq. 8)."""
    lx = (np.roll(p, -1, axis=2) - 2.0 * p + np.roll(p, 1, axis=2)) / g.dx ** 2
    lz = (np.roll(p, -1, axis=1) - 2.0 * p + np.roll(p, 1, axis=1)) / g.dz ** 2
    flux = np.zeros((g.ny + 1,) + p.shape[1:])
    flux[1:g.ny] = (p[1:] - p[:-1]) / g.h[1:g.ny, None, None]
    ly = (flux[1:] - flux[:-1]) / g.dy[:, None, None]
    return lx + ly + lz


def divergence_T(g: Grid, q):
    """Transpose of ``divergence`` (Euclidean inner products): cell field -> (gu, gv, gw)."""
    gu = (np.roll(q, 1, axis=2) - q) / g.dx
    gw = (np.roll(q, 1, axis=1) - q) / g.dz
    qs = q / g.dy[:, None, None]
    gv = np.zeros((g.ny + 1,) + q.shape[1:])
    gv[1:] += qs
    gv[:-1] -= qs
    return gu, gv, gw


def gradient_T(g: Grid, gx, gy, gz):
    """Transpose of ``gradient``: face fields -> cell field (wall entries of gy ignored)."""
    tx = (gx - np.roll(gx, -1, axis=2)) / g.dx
    tz = (gz - np.roll(gz, -1, axis=1)) / g.dz
    s = np.zeros((g.ny + 1,) + gx.shape[1:])
    s[1:g.ny] = gy[1:g.ny] / g.h[1:g.ny, None, None]
    ty = s[:-1] - s[1:]
    return tx + ty + tz
