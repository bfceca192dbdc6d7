"""Pins of the oracle's momentum right-hand side and RK2 timestep (Sec. 2, Eqs. 3-7).

Closed forms of the central staggered differences on chosen fields (a single x or z mode,
the laminar profile, a parabolic wall-normal v), telescoping and kinetic-energy conservation
of the divergence-form advection for divergence-free fields, self-adjointness and sign of the
diffusion operator in the volume inner product, and Heun's scheme against the second-order
Taylor polynomial of exp(dt A) for a linear (advection-free) state.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle.momentum import momentum_rhs, rk2_predictor, timestep

NU = 1.0 / 550.0


def _grid(nx, ny, nz, stretch=None):
    faces = W.uniform_faces(ny) if stretch is None else W.tanh_faces(ny, stretch)
    return oracle.Grid(nx, nz, faces)


def _zeros(g):
    return (np.zeros((g.ny, g.nz, g.nx)), np.zeros((g.ny + 1, g.nz, g.nx)), np.zeros((g.ny, g.nz, g.nx)))


def test_x_mode_advection_and_diffusion_closed_form():
    # u = sin(kappa x) at the x-faces x_i = i dx, v = w = 0: the central flux difference of u^2
    # is cos^2(kappa dx/2) sin(kappa dx)/dx sin(2 kappa x_i); the x-diffusion is the modified
    # wavenumber -4/dx^2 sin^2(kappa dx/2); the no-slip wall rows lose 2 u / dy^2.
    g = _grid(24, 6, 4, stretch=1.7)
    u, v, w = _zeros(g)
    kappa = 2.0 * math.pi * 3 / g.lx
    x = np.arange(g.nx) * g.dx
    u[:] = np.sin(kappa * x)
    ru, rv, rw = momentum_rhs(g, u, v, w, NU, 0.0)
    adv = math.cos(kappa * g.dx / 2) ** 2 * math.sin(kappa * g.dx) / g.dx * np.sin(2 * kappa * x)
    lap = -4.0 / g.dx ** 2 * math.sin(kappa * g.dx / 2) ** 2 * np.sin(kappa * x)
    want = np.broadcast_to(-adv + NU * lap, u.shape).copy()
    want[0] -= NU * 2.0 / g.dy[0] ** 2 * np.sin(kappa * x)
    want[-1] -= NU * 2.0 / g.dy[-1] ** 2 * np.sin(kappa * x)
    assert np.max(np.abs(ru - want)) <= 1e-12 * np.max(np.abs(want))
    assert np.max(np.abs(rv)) == 0.0 and np.max(np.abs(rw)) == 0.0


def test_z_mode_advection_closed_form():
    g = _grid(4, 6, 20, stretch=1.2)
    u, v, w = _zeros(g)
    kappa = 2.0 * math.pi * 2 / g.lz
    z = np.arange(g.nz) * g.dz
    w[:] = np.cos(kappa * z)[None, :, None]
    ru, rv, rw = momentum_rhs(g, u, v, w, 0.0, 0.0)
    # cos^2 a - cos^2 b = -sin(a + b) sin(a - b)
    adv = -math.cos(kappa * g.dz / 2) ** 2 * math.sin(kappa * g.dz) / g.dz * np.sin(2 * kappa * z)
    assert np.max(np.abs(rw - (-adv)[None, :, None])) <= 1e-12 * np.max(np.abs(adv))
    assert np.max(np.abs(ru)) == 0.0 and np.max(np.abs(rv)) == 0.0


def test_laminar_profile_is_steady_except_the_wall_rows():
    # u = 1 - yc^2 on uniform faces with f_x = 2 nu: interior rows are exactly steady (the
    # three-point Laplacian of a quadratic is exact); the no-slip wall rows see the one-sided
    # wall gradient (u_0 - 0)/(dy/2) = 2 - dy/2, so L u = -3/2 there and R_u = nu / 2.
    g = _grid(8, 16, 6)
    u, v, w = _zeros(g)
    u[:] = (1.0 - g.yc ** 2)[:, None, None]
    ru, rv, rw = momentum_rhs(g, u, v, w, NU, 2.0 * NU)
    assert np.max(np.abs(ru[1:-1])) <= 1e-12
    assert np.max(np.abs(ru[0] - 0.5 * NU)) <= 1e-12 and np.max(np.abs(ru[-1] - 0.5 * NU)) <= 1e-12
    assert np.max(np.abs(rv)) == 0.0 and np.max(np.abs(rw)) == 0.0


def test_parabolic_v_closed_form():
    # v = 1 - y^2 at the y-faces (zero on both walls), uniform grid: vcc_j = 1 - yc_j^2 - dy^2/4,
    # so the face difference of vcc^2 over dy is -2 y_f (2 - 2 y_f^2 - dy^2); diffusion is -2 nu.
    g = _grid(4, 12, 4)
    u, v, w = _zeros(g)
    y = g.faces
    v[:] = (1.0 - y ** 2)[:, None, None]
    ru, rv, rw = momentum_rhs(g, u, v, w, NU, 0.0)
    dy = g.dy[0]
    yf = y[1:-1]
    want = 2.0 * yf * (2.0 - 2.0 * yf ** 2 - dy ** 2) - 2.0 * NU
    assert np.max(np.abs(rv[1:-1] - want[:, None, None])) <= 1e-12 * np.max(np.abs(want))
    assert np.max(np.abs(rv[0])) == 0.0 and np.max(np.abs(rv[-1])) == 0.0
    assert np.max(np.abs(ru)) == 0.0 and np.max(np.abs(rw)) == 0.0


@pytest.mark.parametrize("stretch", [None, 2.0])
def test_advection_is_conservative(stretch):
    # Divergence form: the volume integrals of the u and w tendencies telescope to zero (no flux
    # through the no-slip walls), for arbitrary fields.  v's control volumes (height h_f) leave
    # the momentum flux v^2 at the two wall-adjacent cell centres, where v = v_1/2 and v_{Ny-1}/2.
    g = _grid(10, 8, 6, stretch)
    u, v, w = W.random_velocity(11, g.nx, g.ny, g.nz, walls_zero=True)
    ru, rv, rw = momentum_rhs(g, u, v, w, 0.0, 0.0)
    vol = g.dy[:, None, None]
    scale = np.max(np.abs(ru)) * u.size
    assert abs(np.sum(vol * ru)) <= 1e-13 * scale
    assert abs(np.sum(vol * rw)) <= 1e-13 * scale
    vsum = np.sum(g.h[1:-1, None, None] * rv[1:-1])
    boundary = -np.sum((0.5 * v[-2]) ** 2 - (0.5 * v[1]) ** 2)
    assert abs(vsum - boundary) <= 1e-13 * np.max(np.abs(rv)) * v.size


@pytest.mark.parametrize("stretch", [None, 1.8])
def test_advection_conserves_kinetic_energy_for_divergence_free_fields(stretch):
    # The second-order divergence-form scheme on a staggered grid conserves the discrete kinetic
    # energy when the velocity is discretely divergence-free (Morinishi et al., J. Comput. Phys.
    # 143, 1998): sum(dy u N_u) + sum(h v N_v) + sum(dy w N_w) = 0.  A wrong average, index or
    # transposed operand in any flux breaks it.
    g = _grid(12, 10, 8, stretch)
    u, v, w = W.random_velocity(12, g.nx, g.ny, g.nz, walls_zero=True)
    u, v, w, _ = oracle.project(g, u, v, w, 1.0)
    assert np.max(np.abs(oracle.divergence(g, u, v, w))) < 1e-11
    ru, rv, rw = momentum_rhs(g, u, v, w, 0.0, 0.0)
    e = (np.sum(g.dy[:, None, None] * u * ru) + np.sum(g.h[1:-1, None, None] * v[1:-1] * rv[1:-1])
         + np.sum(g.dy[:, None, None] * w * rw))
    scale = np.sum(g.dy[:, None, None] * np.abs(u * ru)) + np.sum(g.dy[:, None, None] * np.abs(w * rw))
    if stretch is None:
        assert abs(e) <= 1e-13 * scale
    else:
        # arithmetic (not distance-weighted) averages across stretched y-faces: not exactly
        # conservative; the defect stays a small fraction of the terms (5.5e-4 here)
        assert abs(e) <= 5e-3 * scale


def _diffusion_only(g, comp):
    """Matrix of the diffusion operator of one component (advection removed by linearity)."""
    def op(x):
        u, v, w = _zeros(g)
        (u, v, w)[comp][...] = x
        r = momentum_rhs(g, u, v, w, 1.0, 0.0)
        # advection is quadratic and diffusion linear: R(x) - R(-x) = 2 L x
        rm = momentum_rhs(g, *((-a) for a in (u, v, w)), 1.0, 0.0)
        return 0.5 * (r[comp] - rm[comp])
    shape = (g.ny + 1, g.nz, g.nx) if comp == 1 else (g.ny, g.nz, g.nx)
    n = int(np.prod(shape))
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        cols.append(op(e.reshape(shape)).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_diffusion_is_self_adjoint_and_negative_in_the_volume_inner_product(comp):
    g = _grid(4, 6, 4, stretch=1.6)
    A = _diffusion_only(g, comp)
    if comp == 1:
        wts = np.concatenate([[0.0], g.h[1:-1], [0.0]])
        keep = np.repeat(wts > 0, g.nz * g.nx)
        A = A[np.ix_(keep, keep)]
        wts = np.repeat(wts[wts > 0], g.nz * g.nx)
    else:
        wts = np.repeat(g.dy, g.nz * g.nx)
    S = wts[:, None] * A
    assert np.max(np.abs(S - S.T)) <= 1e-12 * np.max(np.abs(S))
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    assert ev.max() <= 1e-9 * np.max(np.abs(ev))
    if comp != 1:
        assert ev.max() < 0.0     # no-slip walls: definite (no constant null vector)


def test_heun_matches_second_order_taylor_for_a_linear_state():
    # u = U(y), v = w = 0 stays advection-free, so R(u) = A u + b is affine and Heun's step is
    # u + dt (A u + b) + dt^2/2 A (A u + b).
    g = _grid(4, 8, 4, stretch=1.4)
    rng = np.random.default_rng(3)
    U = rng.standard_normal(g.ny)
    u, v, w = _zeros(g)
    u[:] = U[:, None, None]
    dt, fx = 3e-3, 0.7
    us, vs, ws = rk2_predictor(g, u, v, w, dt, NU, fx)
    # A restricted to y-profiles, by brute force on unit vectors
    A = np.zeros((g.ny, g.ny))
    for k in range(g.ny):
        e = np.zeros((g.ny, g.nz, g.nx))
        e[k] = 1.0
        A[:, k] = momentum_rhs(g, e, v, w, NU, 0.0)[0][:, 0, 0]
    r0 = A @ U + fx
    want = U + dt * r0 + 0.5 * dt * dt * (A @ r0)
    assert np.max(np.abs(us[:, 0, 0] - want)) <= 1e-14 * np.max(np.abs(want))
    assert np.max(np.abs(us - us[:, :1, :1])) == 0.0
    assert np.max(np.abs(vs)) == 0.0 and np.max(np.abs(ws)) == 0.0


def test_timestep_is_divergence_free_and_keeps_the_walls():
    case = W.ChannelCase("t", 16, 12, 8, 2.0)
    g = oracle.Grid(case.nx, case.nz, W.tanh_faces(case.ny, case.stretch))
    u, v, w = W.poiseuille_plus_noise(1, case)
    u1, v1, w1, _ = timestep(g, u, v, w, 1e-4, NU, 2.0 * NU)
    assert np.max(np.abs(oracle.divergence(g, u1, v1, w1))) <= 1e-12 * np.max(np.abs(u)) / 1e-4
    assert np.max(np.abs(v1[0])) == 0.0 and np.max(np.abs(v1[-1])) == 0.0
    # one small step moves the state by O(dt |R|)
    assert 0.0 < np.max(np.abs(u1 - u)) < 0.2
