"""Tridiagonal solvers of Sec. 2.1 (Thomas) and Sec. 2.2 (PDD, Eqs. 10-21).

Test infrastructure only (see the package docstring).

All solvers take the system along axis 0:
    lower[j] x[j-1] + diag[j] x[j] + upper[j] x[j+1] = rhs[j],  j = 0..n-1,
with ``lower[0]`` and ``upper[n-1]`` ignored.  Trailing axes are independent systems
(broadcasting), so one call solves a whole batch of (kx, kz) modes.
"""
from __future__ import annotations

import numpy as np

EXT = np.longdouble          # 64-bit mantissa on x86-64, IEEE quad on aarch64


def _ext(a):
    a = np.asarray(a)
    return a.astype(np.clongdouble if np.iscomplexobj(a) else EXT)


def thomas(lower, diag, upper, rhs, ext: bool = True):
    """Textbook Thomas algorithm (forward elimination, back substitution), Sec. 2.1.

    With ``ext`` the recurrence runs in ``numpy.longdouble`` so its rounding error sits far
    below FP64 even on the weakly dominant low modes; the result is returned in FP64.
    """
    cvt = _ext if ext else np.asarray
    lo, di, up, d = cvt(lower), cvt(diag), cvt(upper), cvt(rhs)
    n = d.shape[0]
    shape = np.broadcast(lo[0], di[0], up[0], d[0]).shape
    cp = np.empty((n,) + shape, dtype=np.result_type(lo, di, up))
    dp = np.empty((n,) + shape, dtype=np.result_type(lo, di, up, d))
    cp[0] = up[0] / di[0]
    dp[0] = d[0] / di[0]
    for j in range(1, n):
        den = di[j] - lo[j] * cp[j - 1]
        cp[j] = up[j] / den
        dp[j] = (d[j] - lo[j] * dp[j - 1]) / den
    x = np.empty_like(dp)
    x[n - 1] = dp[n - 1]
    for j in range(n - 2, -1, -1):
        x[j] = dp[j] - cp[j] * x[j + 1]
    out = np.complex128 if np.iscomplexobj(x) else np.float64
    return x.astype(out)


def pdd(lower, diag, upper, rhs, parts: int, truncated: bool = False):
    """Parallel diagonal dominant algorithm, Sec. 2.2, for a single system (1-D arrays).

    The matrix is split as A = A~ + V E^T (Eqs. 11-14) into ``parts`` diagonal blocks of
    m = n / parts rows.  Following the five-step procedure:

    1-2. every block solves A_i [x~, v, w] = [d^i, a_1^i e_1, c_m^i e_m] (Eq. 20) by Thomas;
    3-4. the interface system Z y = E^T x~ (Eqs. 18, 21) is solved -- exactly (dense, with
         the framed coupling entries) by default, or, with ``truncated``, with v_m^i and w_1^i
         dropped so that Z splits into (parts-1) independent 2x2 systems solved by Cramer's rule;
    5.   x^i = x~^i - v^i y_1^{i-1} - w^i y_2^i (Eq. 19).
    """
    lower = np.asarray(lower, dtype=np.float64)
    diag = np.asarray(diag, dtype=np.float64)
    upper = np.asarray(upper, dtype=np.float64)
    rhs = np.asarray(rhs)
    n = diag.size
    if n % parts:
        raise ValueError("PDD needs parts | n (n = p m, Sec. 2.2)")
    m = n // parts
    dt = np.complex128 if np.iscomplexobj(rhs) else np.float64
    xt = np.zeros(n, dtype=dt)
    v = np.zeros(n)
    w = np.zeros(n)
    for i in range(parts):
        s = slice(i * m, (i + 1) * m)
        lo, di, up = lower[s].copy(), diag[s], upper[s].copy()
        a1, cm = lo[0], up[-1]          # the framed entries of Eq. 12 for this block
        lo[0] = 0.0
        up[-1] = 0.0
        xt[s] = thomas(lo, di, up, rhs[s])
        if i > 0:
            e1 = np.zeros(m)
            e1[0] = a1
            v[s] = thomas(lo, di, up, e1)
        if i < parts - 1:
            em = np.zeros(m)
            em[-1] = cm
            w[s] = thomas(lo, di, up, em)
    k = 2 * (parts - 1)
    if k == 0:
        return xt
    # unknowns y = (y_1^1, y_2^1, y_1^2, y_2^2, ...) with y_1^i <-> row i*m-1 (last of block i)
    # and y_2^i <-> row i*m (first of block i+1), i = 1..parts-1 (1-based block numbers).
    Z = np.eye(k)
    rhs_z = np.zeros(k, dtype=dt)
    for i in range(1, parts):
        r1, r2 = 2 * (i - 1), 2 * (i - 1) + 1
        last_i, first_next = i * m - 1, i * m
        rhs_z[r1] = xt[last_i]
        rhs_z[r2] = xt[first_next]
        # row r1 is E^T Y at row last_i: w^i (column of y_2^i) and v^i (column of y_1^{i-1})
        Z[r1, r2] = w[last_i]
        if i > 1 and not truncated:
            Z[r1, r1 - 2] = v[last_i]           # framed v_m^i
        # row r2 at row first_next: v^{i+1} (column y_1^i) and w^{i+1} (column y_2^{i+1})
        Z[r2, r1] = v[first_next]
        if i < parts - 1 and not truncated:
            Z[r2, r2 + 2] = w[first_next]       # framed w_1^{i+1}
    if truncated:
        y = np.zeros(k, dtype=dt)
        for i in range(1, parts):
            r1, r2 = 2 * (i - 1), 2 * (i - 1) + 1
            det = 1.0 - Z[r1, r2] * Z[r2, r1]
            y[r1] = (rhs_z[r1] - Z[r1, r2] * rhs_z[r2]) / det
            y[r2] = (rhs_z[r2] - Z[r2, r1] * rhs_z[r1]) / det
    else:
        y = np.linalg.solve(Z, rhs_z)
    x = xt.copy()
    for i in range(parts):
        s = slice(i * m, (i + 1) * m)
        if i > 0:
            x[s] -= v[s] * y[2 * (i - 1)]       # y_1^{i-1}
        if i < parts - 1:
            x[s] -= w[s] * y[2 * i + 1]         # y_2^i
    return x
