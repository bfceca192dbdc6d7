"""Pins of the CPU oracle against mathematics that is independent of the oracle itself.

Each test fixes a property that a plausible mistake in the oracle (a dropped term, a wrong
sign or index, a transposed operand) would break: closed-form eigenpairs of the discrete
operator, dense LU solves of the assembled operator, second-order convergence to a
continuous solution on the stretched grid, brute-force transposes, and invariants.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _grid(nx, ny, nz, stretch=None):
    faces = W.uniform_faces(ny) if stretch is None else W.tanh_faces(ny, stretch)
    return oracle.Grid(nx, nz, faces)


def _dense(op, shape_in, shape_out=None):
    """Matrix of a linear map by applying it to unit vectors (brute force)."""
    n = int(np.prod(shape_in))
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        cols.append(np.asarray(op(e.reshape(shape_in))).ravel())
    return np.stack(cols, axis=1)


# --------------------------------------------------------------------------- tridiagonal

def _tri_dense(lo, di, up):
    n = di.size
    A = np.diag(di).astype(float)
    A[np.arange(1, n), np.arange(n - 1)] = lo[1:]
    A[np.arange(n - 1), np.arange(1, n)] = up[:-1]
    return A


def _mp_solve(lo, di, up, d):
    """Reference solve of a tridiagonal system in 40-digit arithmetic (mpmath LU)."""
    import mpmath
    mpmath.mp.dps = 40
    A = mpmath.matrix(_tri_dense(lo, di, up).tolist())
    re = mpmath.lu_solve(A, mpmath.matrix(np.real(d).tolist()))
    im = mpmath.lu_solve(A, mpmath.matrix(np.imag(d).tolist()))
    return np.array([complex(float(re[i]), float(im[i])) for i in range(len(d))])


@pytest.mark.parametrize("sigma", [0.0, 1.0, 1e3, 1e6])
def test_thomas_matches_high_precision_lu_on_channel_rows(sigma):
    g = _grid(8, 48, 8, stretch=2.0)
    a, c = g.lower, g.upper
    di = -(a + c) - sigma
    if sigma == 0.0:
        di[0] -= 1.0        # make the Neumann operator nonsingular for this check
    rng = np.random.default_rng(1)
    d = rng.standard_normal(48) + 1j * rng.standard_normal(48)
    x = oracle.thomas(a, di, c, d)
    ref = _mp_solve(a, di, c, d)
    assert np.max(np.abs(x - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_thomas_batched_broadcast_matches_loop():
    rng = np.random.default_rng(2)
    n, b = 12, 5
    lo = rng.uniform(0.1, 1.0, n)
    up = rng.uniform(0.1, 1.0, n)
    di = -(lo + up)[:, None] - rng.uniform(0.5, 2.0, (1, b))
    d = rng.standard_normal((n, b))
    X = oracle.thomas(lo[:, None], di, up[:, None], d)
    for k in range(b):
        ref = np.linalg.solve(_tri_dense(lo, di[:, k], up), d[:, k])
        assert np.allclose(X[:, k], ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("parts", [1, 2, 4, 8])
@pytest.mark.parametrize("sigma", [1.0, 50.0, 1e4])
def test_pdd_exact_equals_dense(parts, sigma):
    g = _grid(8, 48, 8, stretch=2.0)
    a, c = g.lower, g.upper
    di = -(a + c) - sigma
    rng = np.random.default_rng(3)
    d = rng.standard_normal(48) + 1j * rng.standard_normal(48)
    x = oracle.pdd(a, di, c, d, parts)
    ref = np.linalg.solve(_tri_dense(a, di, c), d)
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_pdd_truncated_is_exact_only_when_coupling_decays():
    # Strongly dominant rows: the framed terms of Eq. 21 are below rounding -> exact.
    n, parts = 96, 4
    lo = np.ones(n)
    up = np.ones(n)
    di = np.full(n, -6.0)
    d = np.random.default_rng(4).standard_normal(n)
    ref = np.linalg.solve(_tri_dense(lo, di, up), d)
    xt = oracle.pdd(lo, di, up, d, parts, truncated=True)
    assert np.max(np.abs(xt - ref)) <= 1e-13 * np.max(np.abs(ref))
    # Weak dominance (the stretched channel's lowest mode): dropping them is visibly wrong,
    # and the exact reduced system repairs it.
    g = _grid(8, 96, 8, stretch=2.0)
    a, c = g.lower, g.upper
    di = -(a + c) - 1.0
    ref = np.linalg.solve(_tri_dense(a, di, c), d)
    xt = oracle.pdd(a, di, c, d, parts, truncated=True)
    xe = oracle.pdd(a, di, c, d, parts, truncated=False)
    assert np.max(np.abs(xt - ref)) > 1e-3 * np.max(np.abs(ref))
    assert np.max(np.abs(xe - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_pdd_rejects_non_divisible_partition():
    with pytest.raises(ValueError):
        oracle.pdd(np.ones(10), -3 * np.ones(10), np.ones(10), np.ones(10), 3)


# --------------------------------------------------------------------------- operators

def test_uniform_grid_closed_form_eigenfunction():
    """cos modes at cell centres are eigenvectors of L_h with modified wavenumbers."""
    nx, ny, nz = 16, 12, 8
    g = _grid(nx, ny, nz)
    mx, my, mz = 3, 2, 1
    x = (np.arange(nx) + 0.5) * g.dx
    z = (np.arange(nz) + 0.5) * g.dz
    yc = -1.0 + (np.arange(ny) + 0.5) * (2.0 / ny)
    p = (np.cos(my * np.pi * (yc + 1.0) / 2.0)[:, None, None]
         * np.cos(2 * np.pi * mz * z / g.lz)[None, :, None]
         * np.cos(2 * np.pi * mx * x / g.lx)[None, None, :])
    dy = 2.0 / ny
    lam = (-(4 / g.dx ** 2) * math.sin(math.pi * mx / nx) ** 2
           - (4 / g.dz ** 2) * math.sin(math.pi * mz / nz) ** 2
           - (4 / dy ** 2) * math.sin(math.pi * my / (2 * ny)) ** 2)
    assert np.allclose(oracle.laplacian(g, p), lam * p, rtol=0, atol=1e-11 * abs(lam))
    sol = oracle.solve(g, lam * p)
    assert np.max(np.abs(sol - p)) <= 1e-13


def test_divergence_of_gradient_is_the_laplacian():
    g = _grid(6, 10, 8, stretch=1.7)
    p = W.random_field(5, (10, 8, 6))
    gx, gy, gz = oracle.gradient(g, p)
    assert np.allclose(oracle.divergence(g, gx, gy, gz), oracle.laplacian(g, p), rtol=0, atol=1e-10)


def test_laplacian_invariants_stretched():
    g = _grid(6, 10, 8, stretch=1.7)
    rng = np.random.default_rng(6)
    p, q = rng.standard_normal((2, 10, 8, 6))
    Wt = g.dy[:, None, None]
    # W L_h is symmetric (finite-volume form)
    assert abs(np.sum(q * Wt * oracle.laplacian(g, p)) - np.sum(p * Wt * oracle.laplacian(g, q))) < 1e-9
    # constants are in the null space; the weighted sum telescopes to zero (no wall flux)
    assert np.max(np.abs(oracle.laplacian(g, np.full((10, 8, 6), 3.0)))) < 1e-10
    assert abs(np.sum(Wt * oracle.laplacian(g, p))) < 1e-9


def test_transposes_are_brute_force_transposes():
    nx, ny, nz = 4, 5, 3
    g = _grid(nx, ny, nz, stretch=1.3)
    cs, vs = (ny, nz, nx), (ny + 1, nz, nx)
    n_c, n_v = ny * nz * nx, (ny + 1) * nz * nx

    def split(vec):
        return vec[:n_c].reshape(cs), vec[n_c:n_c + n_v].reshape(vs), vec[n_c + n_v:].reshape(cs)

    def D(vec):
        return oracle.divergence(g, *split(vec.ravel()))

    def DT(q):
        return np.concatenate([a.ravel() for a in oracle.divergence_T(g, q)])

    def G(p):
        return np.concatenate([a.ravel() for a in oracle.gradient(g, p)])

    def GT(vec):
        return oracle.gradient_T(g, *split(vec.ravel()))

    n_f = 2 * n_c + n_v
    assert np.allclose(_dense(DT, cs), _dense(D, (n_f,)).T, atol=1e-12)
    assert np.allclose(_dense(GT, (n_f,)), _dense(G, cs).T, atol=1e-12)


# --------------------------------------------------------------------------- the solve

@pytest.mark.parametrize("shape,stretch", [((4, 6, 4), 1.5), ((6, 8, 6), 2.0), ((6, 5, 4), None)])
def test_solve_matches_bordered_dense_lu(shape, stretch):
    nx, ny, nz = shape
    g = _grid(nx, ny, nz, stretch)
    cs = (ny, nz, nx)
    L = _dense(lambda p: oracle.laplacian(g, p), cs)
    wts = np.broadcast_to(g.dy[:, None, None], cs).ravel()
    n = L.shape[0]
    B = np.zeros((n + 1, n + 1))
    B[:n, :n] = L
    B[:n, n] = 1.0
    B[n, :n] = wts
    f = W.random_field(7, cs)
    fc = f - np.sum(wts * f.ravel()) / wts.sum()
    rhs = np.concatenate([fc.ravel(), [0.0]])
    ref = np.linalg.solve(B, rhs)[:n].reshape(cs)
    p = oracle.solve(g, f)
    assert np.max(np.abs(p - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_mode00_prefix_sum_closed_form():
    """The (0, 0) profile equals the flux prefix sum: q_{j+1/2} = sum dy F, p_{j+1} = p_j + h q."""
    nx, ny, nz = 4, 24, 4
    g = _grid(nx, ny, nz, stretch=2.0)
    prof = W.random_field(8, ny)
    f = np.broadcast_to(prof[:, None, None], (ny, nz, nx)).copy()
    p = oracle.solve(g, f)
    fc = prof - np.sum(g.dy * prof) / g.dy.sum()
    q = np.cumsum(g.dy * fc)                      # flux through the top face of each cell
    ref = np.zeros(ny)
    for j in range(ny - 1):
        ref[j + 1] = ref[j] + (g.yc[j + 1] - g.yc[j]) * q[j]
    ref -= np.sum(g.dy * ref) / g.dy.sum()
    assert abs(q[-1]) < 1e-12
    assert np.max(np.abs(p - ref[:, None, None])) <= 1e-12 * np.max(np.abs(ref))


def test_constant_rhs_gives_zero_and_linearity_and_shifts():
    g = _grid(8, 12, 6, stretch=1.5)
    cs = (12, 6, 8)
    assert np.max(np.abs(oracle.solve(g, np.full(cs, 2.5)))) < 1e-13
    f1, f2 = W.random_field(9, cs), W.random_field(10, cs)
    p1, p2 = oracle.solve(g, f1), oracle.solve(g, f2)
    assert np.allclose(oracle.solve(g, 2 * f1 - 3 * f2), 2 * p1 - 3 * p2, atol=1e-12)
    assert np.allclose(oracle.solve(g, np.roll(f1, 3, axis=2)), np.roll(p1, 3, axis=2), atol=1e-12)
    assert np.allclose(oracle.solve(g, np.roll(f1, 2, axis=1)), np.roll(p1, 2, axis=1), atol=1e-12)


def _continuous_solution(x, y, z):
    """Solution of lap p = cos(x) cos(4z) cos(pi y/2), dp/dy = 0 at y = +-1, zero mean."""
    k2 = 17.0
    K = math.pi ** 2 / 4 + k2
    A = -(math.pi / 2) / (K * math.sqrt(k2) * math.sinh(math.sqrt(k2)))
    return (np.cos(x)[None, None, :] * np.cos(4 * z)[None, :, None]
            * (-np.cos(np.pi * y / 2) / K + A * np.cosh(math.sqrt(k2) * y))[:, None, None])


def test_second_order_convergence_to_continuous_solution_on_stretched_grid():
    errs = []
    for n in (16, 32, 64):
        g = _grid(n, n, n, stretch=1.5)
        f = W.manufactured_rhs(n, n, n, g.faces)
        x = (np.arange(n) + 0.5) * g.dx
        z = (np.arange(n) + 0.5) * g.dz
        p = oracle.solve(g, f)
        errs.append(np.max(np.abs(p - _continuous_solution(x, g.yc, z))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < o < 2.3 for o in orders), (errs, orders)


def test_residual_of_random_divergence_rhs():
    case = W.CHANNEL_32
    g = oracle.Grid(case.nx, case.nz, W.tanh_faces(case.ny, case.stretch))
    u, v, w = W.random_velocity(0, case.nx, case.ny, case.nz)
    f = oracle.divergence(g, u, v, w)
    p = oracle.solve(g, f)
    r = oracle.residual(g, p, f)
    assert np.max(np.abs(r)) <= 1e-12 * np.max(np.abs(f))
    assert abs(np.einsum("j,jki->", g.dy, p)) < 1e-10


# --------------------------------------------------------------------------- projection

def test_projection_is_divergence_free_idempotent_and_dt_free():
    g = _grid(8, 12, 6, stretch=1.8)
    u, v, w = W.random_velocity(11, 8, 12, 6, walls_zero=True)
    u1, v1, w1, p = oracle.project(g, u, v, w, dt=1e-3)
    div0 = np.max(np.abs(oracle.divergence(g, u, v, w)))
    assert np.max(np.abs(oracle.divergence(g, u1, v1, w1))) <= 1e-12 * div0
    u2, v2, w2, _ = oracle.project(g, u1, v1, w1, dt=0.5)
    assert np.allclose(u2, u1, atol=1e-12) and np.allclose(v2, v1, atol=1e-12)
    assert np.allclose(w2, w1, atol=1e-12)
    assert np.array_equal(v1[0], v[0]) and np.array_equal(v1[-1], v[-1])


def test_projection_with_wall_flux_leaves_only_the_mean_divergence():
    g = _grid(8, 12, 6, stretch=1.8)
    u, v, w = W.random_velocity(12, 8, 12, 6)
    u1, v1, w1, _ = oracle.project(g, u, v, w, dt=1.0)
    d1 = oracle.divergence(g, u1, v1, w1)
    assert np.max(np.abs(d1 - d1.mean())) <= 1e-11 * np.max(np.abs(oracle.divergence(g, u, v, w)))


def test_solve_transposed_is_the_transpose_of_solve():
    g = _grid(6, 7, 4, stretch=1.6)
    cs = (7, 4, 6)
    S = _dense(lambda f: oracle.solve(g, f), cs)
    ST = _dense(lambda r: oracle.solve_transposed(g, r), cs)
    assert np.max(np.abs(ST - S.T)) <= 1e-12 * np.max(np.abs(S))


def test_solve_transposed_equals_volume_weighted_solve():
    """S^T r = W S(W^-1 r) with W = diag(dy_j): L_h^T = W L_h W^-1, and the rhs-mean removal and the
    zero-weighted-mean gauge of S transpose into each other (the identity the adjoint solve of the
    library is built on; the oracle computes S^T through the transposed systems instead)."""
    g = _grid(12, 10, 8, stretch=1.9)
    r = np.random.default_rng(21).standard_normal((10, 8, 12))
    dy = g.dy[:, None, None]
    want = oracle.solve_transposed(g, r)
    got = dy * oracle.solve(g, r / dy)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    assert abs(want.sum()) <= 1e-12 * np.abs(want).sum()


def test_projection_adjoint_brute_force_and_dot_product():
    nx, ny, nz = 4, 5, 4
    g = _grid(nx, ny, nz, stretch=1.4)
    cs, vs = (ny, nz, nx), (ny + 1, nz, nx)
    n_c, n_v = ny * nz * nx, (ny + 1) * nz * nx

    def split(vec):
        vec = vec.ravel()
        return vec[:n_c].reshape(cs), vec[n_c:n_c + n_v].reshape(vs), vec[n_c + n_v:].reshape(cs)

    def P(vec):
        a, b, c, _ = oracle.project(g, *split(vec), dt=0.1)
        return np.concatenate([a.ravel(), b.ravel(), c.ravel()])

    def PT(vec):
        return np.concatenate([a.ravel() for a in oracle.project_adjoint(g, *split(vec))])

    n_f = 2 * n_c + n_v
    M, MT = _dense(P, (n_f,)), _dense(PT, (n_f,))
    assert np.max(np.abs(MT - M.T)) < 1e-11
    # larger dot-product test, walls included
    g2 = _grid(8, 10, 6, stretch=1.8)
    d = W.random_velocity(13, 8, 10, 6)
    wgt = W.weight_field(14, 8, 10, 6)
    Pd = oracle.project(g2, *d, dt=1.0)[:3]
    PTw = oracle.project_adjoint(g2, *wgt)
    lhs = sum(np.sum(a * b) for a, b in zip(Pd, wgt))
    rhs = sum(np.sum(a * b) for a, b in zip(d, PTw))
    assert abs(lhs - rhs) <= 1e-12 * sum(np.sum(np.abs(a * b)) for a, b in zip(d, PTw))


# ---------------------------------------------------------------- PDD inside the Poisson solve

@pytest.mark.parametrize("parts", [2, 4, 8])
def test_solve_pdd_exact_equals_the_thomas_solve(parts):
    g = _grid(16, 32, 12, stretch=2.0)
    f = oracle.divergence(g, *W.random_velocity(7, g.nx, g.ny, g.nz))
    want = oracle.solve(g, f)
    got = oracle.solve_pdd(g, f, parts, truncated=False)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_solve_pdd_truncated_two_blocks_has_nothing_to_drop():
    # with two blocks Z is a single 2x2 system: no framed entry exists (Eq. 21)
    g = _grid(16, 32, 12, stretch=2.0)
    f = oracle.divergence(g, *W.random_velocity(8, g.nx, g.ny, g.nz))
    want = oracle.solve(g, f)
    got = oracle.solve_pdd(g, f, 2, truncated=True)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_solve_pdd_truncation_error_decays_with_the_weakest_wavenumber():
    # Sec. 2.2: the dropped entries are the far ends of the spikes, which decay across a block like
    # exp(-sqrt(sigma) L_block); sigma >= (2 pi / L)^2 for the weakest non-(0,0) mode, so with the
    # block length fixed (uniform y, P = 4) shrinking the periodic lengths L drives the truncation
    # error from O(1) to rounding, and the channel's own weak modes keep it large.
    errs = []
    for L in (2 * np.pi, np.pi / 4, np.pi / 32):
        g = oracle.Grid(16, 12, W.uniform_faces(64), lx=L, lz=L)
        f = oracle.divergence(g, *W.random_velocity(9, g.nx, g.ny, g.nz))
        want = oracle.solve(g, f)
        got = oracle.solve_pdd(g, f, 4, truncated=True)
        errs.append(np.max(np.abs(got - want)) / np.max(np.abs(want)))
    assert errs[0] > 0.05 and 1e-4 < errs[1] < 1e-2 and errs[2] < 1e-13
