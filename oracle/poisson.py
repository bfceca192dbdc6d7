"""Pressure Poisson solve and projection (Sec. 2, Eqs. 4, 7, 8, 9), FP64, plain definition.

Test infrastructure only (see the package docstring).

``solve`` returns the exact solution (up to rounding) of the discrete problem
    L_h p = f - <f>,     sum_{ijk} dy_j p_{jki} = 0,
where <f> is the volume-weighted mean (dy_j weights).  It follows Eq. 9: a complex DFT in
each periodic direction over *all* Nx x Nz modes (no half-spectrum symmetry is used), one
wall-normal tridiagonal system per (kx, kz) solved by the Thomas algorithm in extended
precision, the singular (0, 0) mode solved densely with the gauge as a bordering row, and
the inverse DFTs.  The transforms are library FFTs (numpy.fft) used as a step.
"""
from __future__ import annotations

import numpy as np

from .grid import Grid
from .stencils import divergence, gradient, laplacian, divergence_T, gradient_T
from .tridiag import thomas, pdd

_CHUNK = 64          # kz planes per Thomas call (memory only; the systems are independent)


def _weighted_mean(g: Grid, f):
    wsum = g.dy.sum() * g.nx * g.nz
    return float(np.einsum("j,jki->", g.dy, f) / wsum)


def _bordered_mode00(g: Grid, F0, transposed: bool):
    """Solve the singular (0, 0) wall-normal system with a bordering gauge row.

    Forward:  T p = F,  sum_j dy_j p_j = 0     (T = the y-operator; left null vector dy).
    Transposed: T^T q = F, sum_j q_j = 0        (left null vector 1).
    """
    ny = g.ny
    a, c = g.lower, g.upper
    T = np.zeros((ny, ny))
    for j in range(ny):
        T[j, j] = -(a[j] + c[j])
        if j > 0:
            T[j, j - 1] = a[j]
        if j < ny - 1:
            T[j, j + 1] = c[j]
    if transposed:
        T = T.T
        gauge, border = np.ones(ny), g.dy
    else:
        gauge, border = g.dy, np.ones(ny)
    B = np.zeros((ny + 1, ny + 1))
    B[:ny, :ny] = T
    B[:ny, ny] = border
    B[ny, :ny] = gauge
    rhs = np.zeros(ny + 1, dtype=np.complex128)
    rhs[:ny] = F0
    sol = np.linalg.solve(B, rhs)
    return sol[:ny]


def _spectral_solve(g: Grid, F, transposed: bool):
    """Solve every (kx, kz) wall-normal system of Eq. 9 in place of F (Ny, Nz, Nx)."""
    a, c = g.lower, g.upper
    if transposed:      # row j of T^T: sub-diagonal c_{j-1}, super-diagonal a_{j+1}
        lo = np.zeros(g.ny)
        up = np.zeros(g.ny)
        lo[1:] = c[:-1]
        up[:-1] = a[1:]
    else:
        lo, up = a, c
    lam = g.lambda_z()[:, None] + g.lambda_x()[None, :]          # (Nz, Nx)
    P = np.empty_like(F)
    # the (0, 0) system is singular; its Thomas result is discarded and replaced below
    for k0 in range(0, g.nz, _CHUNK):
        k1 = min(g.nz, k0 + _CHUNK)
        diag = -(a + c)[:, None, None] + lam[None, k0:k1, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            P[:, k0:k1, :] = thomas(lo[:, None, None], diag, up[:, None, None], F[:, k0:k1, :])
    P[:, 0, 0] = _bordered_mode00(g, F[:, 0, 0], transposed)
    return P


def solve(g: Grid, f):
    """p with L_h p = f - <f> and zero volume-weighted mean (Eqs. 7-9)."""
    f = np.asarray(f, dtype=np.float64)
    fc = f - _weighted_mean(g, f)
    F = np.fft.fft2(fc, axes=(1, 2))
    P = _spectral_solve(g, F, transposed=False)
    return np.fft.ifft2(P, axes=(1, 2)).real


def solve_pdd(g: Grid, f, parts: int, truncated: bool, exact_modes=None):
    """``solve`` with every wall-normal system of Eq. 9 solved by the PDD algorithm of Sec. 2.2
    (``tridiag.pdd``): with the exact reduced system, or truncated as in the paper (the framed
    coupling entries dropped).  ``exact_modes(kx, kz)`` (signed kx, kz) may name modes that keep
    the exact reduced system.  One mode at a time: for small grids only."""
    f = np.asarray(f, dtype=np.float64)
    fc = f - _weighted_mean(g, f)
    F = np.fft.fft2(fc, axes=(1, 2))
    a, c = g.lower, g.upper
    lamx, lamz = g.lambda_x(), g.lambda_z()
    P = np.empty_like(F)
    for kz in range(g.nz):
        for kx in range(g.nx):
            if kx == 0 and kz == 0:
                continue
            skx = kx if kx <= g.nx // 2 else kx - g.nx
            skz = kz if kz <= g.nz // 2 else kz - g.nz
            trunc = truncated and not (exact_modes is not None and exact_modes(skx, skz))
            diag = -(a + c) + lamx[kx] + lamz[kz]
            P[:, kz, kx] = pdd(a, diag, c, F[:, kz, kx], parts, truncated=trunc)
    P[:, 0, 0] = _bordered_mode00(g, F[:, 0, 0], transposed=False)
    return np.fft.ifft2(P, axes=(1, 2)).real


def solve_transposed(g: Grid, r):
    """S^T r: the transpose of the gauged solve ``solve`` (as a linear map of f).

    With S = Z L_h^+ Pi (Pi f = f - <f>, Z the zero-weighted-mean gauge, both I - 1 omega^T,
    omega_j = dy_j / (Nx Nz sum dy)), S^T r = Pi^T q where q is any solution of
    L_h^T q = Z^T r = r - omega sum(r).  The (0, 0) system is gauged by sum(q) = 0, which is
    already the range of Pi^T, so the final Pi^T only removes rounding.
    """
    r = np.asarray(r, dtype=np.float64)
    omega = g.dy / (g.dy.sum() * g.nx * g.nz)
    rc = r - omega[:, None, None] * r.sum()
    R = np.fft.fft2(rc, axes=(1, 2))
    Q = _spectral_solve(g, R, transposed=True)
    q = np.fft.ifft2(Q, axes=(1, 2)).real
    return q - omega[:, None, None] * q.sum()


def residual(g: Grid, p, f):
    """L_h p - (f - <f>)."""
    f = np.asarray(f, dtype=np.float64)
    return laplacian(g, p) - (f - _weighted_mean(g, f))


def project(g: Grid, u, v, w, dt: float):
    """Eqs. 4 and 7: p solves L_h p = D u*/dt (made compatible); u = u* - dt G p.

    The wall faces of v are boundary values: they enter the divergence and are not changed.
    Returns (u, v, w, p).
    """
    p = solve(g, divergence(g, u, v, w) / dt)
    gx, gy, gz = gradient(g, p)
    return u - dt * gx, v - dt * gy, w - dt * gz, p


def project_adjoint(g: Grid, gu, gv, gw):
    """Transpose of the velocity map u* -> u of ``project`` (the map does not depend on dt).

    The map is P = I - G S D, so P^T = I - D^T S^T G^T (``solve_transposed`` is S^T).
    """
    q = solve_transposed(g, gradient_T(g, gu, gv, gw))
    du, dv, dw = divergence_T(g, q)
    return gu - du, gv - dv, gw - dw
