"""Momentum right-hand side and the RK2 timestep of the projection method (Sec. 2, Eqs. 2-7).

Test infrastructure only (see the package docstring).

R(u) = -N(u) + L(u) + F.  Sec. 2 fixes only second-order central differences on the staggered
grid and Eqs. 3-6; the readings taken here are:
* N(u) = div(u u) in divergence form, face values by arithmetic averages of the two nearest
  nodes (the second-order central scheme on the staggered grid);
* L(u) = nu lap(u): three-point Laplacians; for u and w the wall flux uses the no-slip value 0 at
  the wall, half a cell from the first node: du/dy|wall = (u_0 - 0) / (dy_0 / 2);
* F = (fx, 0, 0): the constant streamwise pressure-gradient forcing that drives the channel
  (Sec. 2); fx = 2 nu keeps u = 1 - y^2 steady in the continuum.
v's wall faces (no penetration) stay fixed.  One step is Heun's RK2 (Eqs. 5-6) followed by one
projection (Eqs. 4, 7): u^{n+1} = P(u*).
"""
from __future__ import annotations

import numpy as np

from .grid import Grid
from .poisson import project


def _xp(a):
    return np.roll(a, -1, axis=2)


def _xm(a):
    return np.roll(a, 1, axis=2)


def _zp(a):
    return np.roll(a, -1, axis=1)


def _zm(a):
    return np.roll(a, 1, axis=1)


def _wall_diffusion_y(g: Grid, q):
    """d/dy(dq/dy) at cell rows for a cell-row field q that vanishes on both walls (no slip)."""
    ny = g.ny
    grad = np.zeros((ny + 1,) + q.shape[1:])
    grad[1:ny] = (q[1:] - q[:-1]) / g.h[1:ny, None, None]
    grad[0] = (q[0] - 0.0) / (0.5 * g.dy[0])
    grad[ny] = (0.0 - q[-1]) / (0.5 * g.dy[-1])
    return (grad[1:] - grad[:-1]) / g.dy[:, None, None]


def momentum_rhs(g: Grid, u, v, w, nu: float, fx: float):
    """(R_u, R_v, R_w) = -N(u) + nu lap(u) + F on the staggered faces; R_v = 0 on the walls."""
    ny = g.ny
    dx, dz = g.dx, g.dz
    dyc = g.dy[:, None, None]
    # ---------------- u at x-faces (j, k, i) ----------------
    uc = 0.5 * (u + _xp(u))                       # u at cell centre i (right of face i)
    adv_x = (uc ** 2 - _xm(uc) ** 2) / dx
    vu = np.zeros((ny + 1,) + u.shape[1:])
    vx = 0.5 * (_xm(v) + v)                       # v at (x-face i, y-face f)
    vu[1:ny] = vx[1:ny] * 0.5 * (u[:-1] + u[1:])
    adv_y = (vu[1:] - vu[:-1]) / dyc
    wx = 0.5 * (_xm(w) + w)                       # w at (x-face i, z-face k)
    wu = wx * 0.5 * (_zm(u) + u)
    adv_z = (_zp(wu) - wu) / dz
    dif = ((_xp(u) - 2 * u + _xm(u)) / dx ** 2 + (_zp(u) - 2 * u + _zm(u)) / dz ** 2 + _wall_diffusion_y(g, u))
    ru = -(adv_x + adv_y + adv_z) + nu * dif + fx
    # ---------------- w at z-faces (j, k, i) ----------------
    wc = 0.5 * (w + _zp(w))
    adv_z = (wc ** 2 - _zm(wc) ** 2) / dz
    uz = 0.5 * (_zm(u) + u)                       # u at (x-face i, z-face k)
    uw = uz * 0.5 * (_xm(w) + w)
    adv_x = (_xp(uw) - uw) / dx
    vw = np.zeros((ny + 1,) + w.shape[1:])
    vz = 0.5 * (_zm(v) + v)                       # v at (y-face f, z-face k)
    vw[1:ny] = vz[1:ny] * 0.5 * (w[:-1] + w[1:])
    adv_y = (vw[1:] - vw[:-1]) / dyc
    dif = ((_xp(w) - 2 * w + _xm(w)) / dx ** 2 + (_zp(w) - 2 * w + _zm(w)) / dz ** 2 + _wall_diffusion_y(g, w))
    rw = -(adv_x + adv_y + adv_z) + nu * dif
    # ---------------- v at y-faces f = 1..ny-1 ----------------
    rv = np.zeros_like(v)
    vi = v[1:ny]
    vcc = 0.5 * (v[:-1] + v[1:])                  # v at cell centres j
    hf = g.h[1:ny, None, None]
    adv_y = (vcc[1:] ** 2 - vcc[:-1] ** 2) / hf
    ux = 0.5 * (u[:-1] + u[1:])                   # u at (x-face i, y-face f)
    uv = ux * 0.5 * (_xm(vi) + vi)
    adv_x = (_xp(uv) - uv) / dx
    wz = 0.5 * (w[:-1] + w[1:])                   # w at (z-face k, y-face f)
    wv = wz * 0.5 * (_zm(vi) + vi)
    adv_z = (_zp(wv) - wv) / dz
    dvy = (v[2:] - v[1:-1]) / g.dy[1:, None, None] - (v[1:-1] - v[:-2]) / g.dy[:-1, None, None]
    dif = (_xp(vi) - 2 * vi + _xm(vi)) / dx ** 2 + (_zp(vi) - 2 * vi + _zm(vi)) / dz ** 2 + dvy / hf
    rv[1:ny] = -(adv_x + adv_y + adv_z) + nu * dif
    return ru, rv, rw


def rk2_predictor(g: Grid, u, v, w, dt: float, nu: float, fx: float):
    """Heun's RK2 (Eqs. 5-6): u_bar = u + dt R(u); u* = u + dt/2 (R(u) + R(u_bar))."""
    r0 = momentum_rhs(g, u, v, w, nu, fx)
    ub = [a + dt * r for a, r in zip((u, v, w), r0)]
    r1 = momentum_rhs(g, *ub, nu, fx)
    return tuple(a + 0.5 * dt * (x + y) for a, x, y in zip((u, v, w), r0, r1))


def timestep(g: Grid, u, v, w, dt: float, nu: float, fx: float):
    """One timestep of the fully explicit projection method: RK2 predictor, then Eqs. 4 and 7.

    Returns (u, v, w, p) at the new time level, p the pressure of the projection."""
    us, vs, ws = rk2_predictor(g, u, v, w, dt, nu, fx)
    return project(g, us, vs, ws, dt)
