"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Tolerances (relative to the largest magnitude of the oracle result):
* FP64 (PP_FP64): 1e-12.
* FP32 (PP_FP32): 2e-5  -- FP32 FFTs (~1e-7 log2 N) and FP32 margin-Thomas (~1e-6 on the
  weakest modes); the lowest modes run in FP64.
* FP32 + refinement (PP_FP32_REFINED): one correction squares the FP32 error
  (eps <= 2e-5 -> eps^2 ~ 4e-10, with an O(1) growth factor): 2e-9; two corrections reach the
  FP64 residual's floor: 1e-12.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


@pytest.fixture(scope="module")
def P():
    from paper_2104_08863_gb300 import build as b
    b.build()
    import paper_2104_08863_gb300 as mod
    return mod


def relerr(got, want):
    return float(np.max(np.abs(np.asarray(got) - want)) / np.max(np.abs(want)))


def to_dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype)


def solve_gpu(P, plan, f, dtype=torch.float64):
    ft = to_dev(f, dtype)
    out = plan.solve(ft)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


# ------------------------------------------------------------------------------ FP64 solve

@pytest.mark.parametrize("rhs", ["manufactured", "random_divergence"])
@pytest.mark.parametrize("tridiag,parts", [(1, 1), (2, 4), (2, 8)])
def test_fp64_solve_channel32(P, rhs, tridiag, parts):
    case = W.CHANNEL_32
    faces = W.tanh_faces(case.ny, case.stretch)
    g = oracle.Grid(case.nx, case.nz, faces)
    if rhs == "manufactured":
        f = W.manufactured_rhs(case.nx, case.ny, case.nz, faces)
    else:
        f = oracle.divergence(g, *W.random_velocity(0, case.nx, case.ny, case.nz))
    want = oracle.solve(g, f)
    plan = P.Plan(case.nx, case.ny, case.nz, faces, precision=P.PP_FP64, tridiag=tridiag, pdd_parts=parts,
                  device=DEV)
    got = solve_gpu(P, plan, f)
    assert relerr(got, want) <= 1e-12


@pytest.mark.parametrize("nx,ny,nz,parts", [
    (4, 2, 2, 1), (6, 6, 3, 3), (12, 10, 9, 5), (24, 12, 18, 4), (48, 16, 27, 16), (96, 24, 12, 6),
    (64, 48, 96, 8), (192, 36, 8, 2), (384, 8, 6, 8), (128, 64, 256, 32), (8, 96, 1536, 3),
])
def test_fp64_solve_ragged_sizes(P, nx, ny, nz, parts):
    faces = W.tanh_faces(ny, 1.7)
    g = oracle.Grid(nx, nz, faces)
    f = W.random_field(21, (ny, nz, nx))
    want = oracle.solve(g, f)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP64, tridiag=P.PT_PDD_EXACT, pdd_parts=parts, device=DEV)
    got = solve_gpu(P, plan, f)
    assert relerr(got, want) <= 1e-12


def test_fp64_solve_in_place_and_repeatable(P):
    nx, ny, nz = 24, 16, 12
    faces = W.tanh_faces(ny, 2.0)
    g = oracle.Grid(nx, nz, faces)
    f = W.random_field(22, (ny, nz, nx))
    want = oracle.solve(g, f)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP64, pdd_parts=2, device=DEV)
    ft = to_dev(f)
    plan.solve(ft, out=ft)
    a = ft.cpu().numpy()
    assert relerr(a, want) <= 1e-12
    b = solve_gpu(P, plan, f)
    assert np.array_equal(b, solve_gpu(P, plan, f))


def test_fp64_closed_form_uniform_grid(P):
    nx, ny, nz = 16, 12, 8
    faces = W.uniform_faces(ny)
    g = oracle.Grid(nx, nz, faces)
    x = (np.arange(nx) + 0.5) * g.dx
    z = (np.arange(nz) + 0.5) * g.dz
    yc = -1.0 + (np.arange(ny) + 0.5) * (2.0 / ny)
    p = (np.cos(2 * np.pi * (yc + 1.0) / 2.0)[:, None, None] * np.cos(2 * np.pi * z / g.lz)[None, :, None]
         * np.cos(2 * np.pi * 3 * x / g.lx)[None, None, :])
    lam = (-(4 / g.dx ** 2) * np.sin(np.pi * 3 / nx) ** 2 - (4 / g.dz ** 2) * np.sin(np.pi / nz) ** 2
           - (4 / (2.0 / ny) ** 2) * np.sin(np.pi * 2 / (2 * ny)) ** 2)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP64, pdd_parts=3, device=DEV)
    got = solve_gpu(P, plan, lam * p)
    assert np.max(np.abs(got - p)) <= 1e-13


def test_fp64_constant_rhs_gives_zero(P):
    nx, ny, nz = 8, 8, 8
    plan = P.Plan(nx, ny, nz, W.tanh_faces(ny, 1.5), precision=P.PP_FP64, device=DEV)
    got = solve_gpu(P, plan, np.full((ny, nz, nx), 3.0))
    assert np.max(np.abs(got)) < 1e-13


# ------------------------------------------------------------------------------ projection

@pytest.mark.parametrize("walls_zero", [True, False])
def test_fp64_projection_channel32(P, walls_zero):
    case = W.CHANNEL_32
    faces = W.tanh_faces(case.ny, case.stretch)
    g = oracle.Grid(case.nx, case.nz, faces)
    u, v, w = W.random_velocity(0, case.nx, case.ny, case.nz, walls_zero=walls_zero)
    dt = 1e-3
    want = oracle.project(g, u, v, w, dt)
    plan = P.Plan(case.nx, case.ny, case.nz, faces, precision=P.PP_FP64, pdd_parts=4, device=DEV)
    ut, vt, wt = to_dev(u), to_dev(v), to_dev(w)
    pt = torch.empty(case.ny, case.nz, case.nx, dtype=torch.float64, device=DEV)
    plan.project(ut, vt, wt, dt, p_out=pt)
    torch.cuda.synchronize()
    for got, ref in zip((ut, vt, wt, pt), want):
        assert relerr(got.cpu().numpy(), ref) <= 1e-12
    assert np.array_equal(vt[0].cpu().numpy(), v[0]) and np.array_equal(vt[-1].cpu().numpy(), v[-1])
    if walls_zero:
        d = oracle.divergence(g, ut.cpu().numpy(), vt.cpu().numpy(), wt.cpu().numpy())
        assert np.max(np.abs(d)) <= 1e-12 * np.max(np.abs(oracle.divergence(g, u, v, w)))


def test_fp64_projection_adjoint_channel(P):
    nx, ny, nz = 24, 16, 12
    faces = W.tanh_faces(ny, 1.8)
    g = oracle.Grid(nx, nz, faces)
    wu, wv, ww = W.weight_field(4, nx, ny, nz)
    want = oracle.project_adjoint(g, wu, wv, ww)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP64, pdd_parts=4, device=DEV)
    gu, gv, gw = to_dev(wu), to_dev(wv), to_dev(ww)
    plan.project_adjoint(gu, gv, gw)
    torch.cuda.synchronize()
    for got, ref in zip((gu, gv, gw), want):
        assert relerr(got.cpu().numpy(), ref) <= 1e-12


# ------------------------------------------------------------------------------ FP32 forms

@pytest.mark.parametrize("nx,ny,nz,parts", [(32, 32, 32, 4), (96, 48, 64, 1), (64, 96, 48, 2)])
def test_fp32_solve(P, nx, ny, nz, parts):
    faces = W.tanh_faces(ny, 2.0)
    g = oracle.Grid(nx, nz, faces)
    f = oracle.divergence(g, *W.random_velocity(2, nx, ny, nz))
    f -= np.einsum("j,jki->", g.dy, f) / (g.dy.sum() * nx * nz)
    want = oracle.solve(g, f)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32, pdd_parts=parts, fp64_low_modes=4, device=DEV)
    got = solve_gpu(P, plan, f, dtype=torch.float32)
    assert relerr(got, want) <= 2e-5


@pytest.mark.parametrize("nx,ny,nz,parts,steps,tol", [
    (32, 32, 32, 4, 1, 2e-9), (96, 48, 64, 2, 1, 2e-9), (64, 96, 48, 4, 2, 1e-12), (64, 96, 48, 4, 3, 1e-12)])
def test_fp32_refined_solve(P, nx, ny, nz, parts, steps, tol):
    faces = W.tanh_faces(ny, 2.2)
    g = oracle.Grid(nx, nz, faces)
    f = oracle.divergence(g, *W.random_velocity(2, nx, ny, nz))
    want = oracle.solve(g, f)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32_REFINED, pdd_parts=parts, fp64_low_modes=4,
                  refine_steps=steps, device=DEV)
    ft = to_dev(f)
    out = torch.empty_like(ft)
    plan.solve(ft, out=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert relerr(got, want) <= tol
    # the gauge (zero dy-weighted mean) holds to FP64 accuracy although the transforms are FP32
    wmean = np.einsum("j,jki->", g.dy, got) / (g.dy.sum() * nx * nz)
    assert abs(wmean) <= 1e-14 * np.max(np.abs(want))


def test_fp32_projection_and_adjoint(P):
    nx, ny, nz = 32, 24, 16
    faces = W.tanh_faces(ny, 1.8)
    g = oracle.Grid(nx, nz, faces)
    u, v, w = W.random_velocity(3, nx, ny, nz)
    want = oracle.project(g, u, v, w, 1e-3)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32, pdd_parts=2, device=DEV)
    ut, vt, wt = (to_dev(a, torch.float32) for a in (u, v, w))
    plan.project(ut, vt, wt, 1e-3)
    for got, ref in zip((ut, vt, wt), want[:3]):
        assert relerr(got.double().cpu().numpy(), ref) <= 2e-5
    wts = W.weight_field(4, nx, ny, nz)
    wantT = oracle.project_adjoint(g, *wts)
    gt = [to_dev(a, torch.float32) for a in wts]
    plan.project_adjoint(*gt)
    for got, ref in zip(gt, wantT):
        assert relerr(got.double().cpu().numpy(), ref) <= 2e-5


# ------------------------------------------------------------------------------ errors

def test_nonfinite_input_sets_device_status(P):
    nx, ny, nz = 8, 8, 8
    plan = P.Plan(nx, ny, nz, W.tanh_faces(ny, 1.5), precision=P.PP_FP64, flags=P.POISSON_CHECK_FINITE,
                  device=DEV)
    f = np.zeros((ny, nz, nx))
    f[3, 2, 1] = np.nan
    plan.solve(to_dev(f))
    assert plan.device_status() == 6
    plan.solve(to_dev(np.ones((ny, nz, nx))))
    assert plan.device_status() == 0


@pytest.mark.parametrize("prec,comp", [(0, "v"), (0, "w"), (1, "v"), (2, "w")])
def test_nonfinite_velocity_component_sets_device_status(P, prec, comp):
    """POISSON_CHECK_FINITE scans every velocity component of the projection, not only u."""
    nx, ny, nz = 16, 8, 8
    plan = P.Plan(nx, ny, nz, W.tanh_faces(ny, 1.5), precision=prec, pdd_parts=2, flags=P.POISSON_CHECK_FINITE,
                  device=DEV)
    dtype = torch.float32 if prec == 1 else torch.float64
    u, v, w = (to_dev(a, dtype) for a in W.random_velocity(7, nx, ny, nz))
    {"v": v, "w": w}[comp][3, 2, 5] = float("nan")
    p = torch.empty(ny, nz, nx, dtype=dtype, device=DEV)
    plan.project(u, v, w, 1e-3, p_out=p)
    assert plan.device_status() == 6
    u, v, w = (to_dev(a, dtype) for a in W.random_velocity(7, nx, ny, nz))
    plan.project(u, v, w, 1e-3, p_out=p)
    assert plan.device_status() == 0


@pytest.mark.parametrize("nx,ny,nz,parts,steps,tol", [(48, 24, 36, 4, 2, 1e-12), (64, 32, 54, 2, 1, 2e-9)])
def test_fp32_refined_projection_matches_oracle(P, nx, ny, nz, parts, steps, tol):
    """projection_step of PP_FP32_REFINED plans: pairs, double-float divergence, refined solve, gradient."""
    faces = W.tanh_faces(ny, 2.0)
    g = oracle.Grid(nx, nz, faces)
    u, v, w = W.random_velocity(8, nx, ny, nz)
    dt = 2e-3
    want = oracle.project(g, u, v, w, dt)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32_REFINED, pdd_parts=parts, fp64_low_modes=4,
                  refine_steps=steps, device=DEV)
    ut, vt, wt = to_dev(u), to_dev(v), to_dev(w)
    pt = plan.project(ut, vt, wt, dt)
    torch.cuda.synchronize()
    for got, ref in zip((ut, vt, wt, pt), want):
        assert relerr(got.cpu().numpy(), ref) <= tol
    # the fields round-trip through FP32 pairs (48-bit significands): the wall faces of v keep
    # their values to 2^-48 relative
    for wall in (0, -1):
        assert np.max(np.abs(vt[wall].cpu().numpy() - v[wall])) <= 2.0 ** -47 * np.max(np.abs(v))
    from paper_2104_08863_gb300 import _native
    L = _native.lib()
    st = torch.cuda.current_stream().cuda_stream
    assert L.projection_step(plan._h, ut.data_ptr(), vt.data_ptr(), wt.data_ptr(), 0, dt, st) == _native.PS_EINVAL
    assert L.projection_step(plan._h, ut.data_ptr(), vt.data_ptr(), wt.data_ptr(), ut.data_ptr(), dt, st) == \
        _native.PS_EINVAL


@pytest.mark.parametrize("prec,tol", [(0, 1e-14), (1, 2e-6), (2, 1e-14)])
def test_divergence_field_matches_oracle(P, prec, tol):
    """poisson_divergence: f = D(u)/dt of Eq. 7 as a field, element by element."""
    nx, ny, nz = 48, 20, 36
    faces = W.tanh_faces(ny, 1.7)
    g = oracle.Grid(nx, nz, faces)
    u, v, w = W.random_velocity(10, nx, ny, nz)
    dt = 3e-3
    want = oracle.divergence(g, u, v, w) / dt
    plan = P.Plan(nx, ny, nz, faces, precision=prec, pdd_parts=2, device=DEV)
    dtype = torch.float32 if prec == 1 else torch.float64
    f = plan.divergence(to_dev(u, dtype), to_dev(v, dtype), to_dev(w, dtype), dt)
    torch.cuda.synchronize()
    assert relerr(f.double().cpu().numpy(), want) <= tol


def test_bad_arguments_are_rejected(P):
    nx, ny, nz = 8, 8, 8
    plan = P.Plan(nx, ny, nz, W.tanh_faces(ny, 1.5), precision=P.PP_FP64, device=DEV)
    with pytest.raises(ValueError):
        plan.solve(torch.zeros((ny, nz, nx), dtype=torch.float32, device=DEV))
    from paper_2104_08863_gb300 import _native
    L = _native.lib()
    buf = torch.zeros(ny * nz * nx + 1, dtype=torch.float64, device=DEV)
    mis = buf.data_ptr() + 8     # not 16-byte aligned
    assert L.poisson_solve(plan._h, mis, mis, torch.cuda.current_stream().cuda_stream) == _native.PS_EINVAL
    assert L.poisson_solve(plan._h, 0, buf.data_ptr(), 0) == _native.PS_EINVAL
    assert L.projection_step(plan._h, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 0, -1.0, 0) == \
        _native.PS_EINVAL


# ------------------------------------------------------------------ truncated PDD (Sec. 2.2)

@pytest.mark.parametrize("parts", [3, 4, 8])
def test_fp64_truncated_pdd_matches_oracle_truncated(P, parts):
    """PT_PDD_TRUNCATED drops the framed coupling entries of Z as the paper does; on the stretched
    channel that changes the weak modes by O(1e-2), and the GPU must reproduce exactly that."""
    nx, ny, nz = 32, 48, 16
    faces = W.tanh_faces(ny, 2.0)
    g = oracle.Grid(nx, nz, faces)
    f = oracle.divergence(g, *W.random_velocity(10, nx, ny, nz))
    want = oracle.solve_pdd(g, f, parts, truncated=True)
    exact = oracle.solve(g, f)
    assert relerr(want, exact) > 1e-4          # the truncation is visible on this grid
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP64, tridiag=P.PT_PDD_TRUNCATED, pdd_parts=parts, device=DEV)
    got = solve_gpu(P, plan, f)
    assert relerr(got, want) <= 1e-12


@pytest.mark.parametrize("parts", [3, 4, 8])
def test_fp32_truncated_pdd_matches_oracle_truncated(P, parts):
    """FP32 truncated PDD (the reduced-system table built without the coupling); the lowest modes
    that the FP32 form solves in FP64 keep the exact reduced system."""
    nx, ny, nz, L = 32, 48, 16, 4
    faces = W.tanh_faces(ny, 2.0)
    g = oracle.Grid(nx, nz, faces)
    f = oracle.divergence(g, *W.random_velocity(11, nx, ny, nz))
    want = oracle.solve_pdd(g, f, parts, truncated=True, exact_modes=lambda kx, kz: abs(kx) <= L and abs(kz) <= L)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32, tridiag=P.PT_PDD_TRUNCATED, pdd_parts=parts,
                  fp64_low_modes=L, device=DEV)
    got = solve_gpu(P, plan, f, dtype=torch.float32)
    assert relerr(got, want) <= 2e-5


def test_fp32_refined_solve_ragged_staged_tiles(P):
    """Nx/2 = 256 takes the x-transform whose FP64 right-hand side is staged by bulk copies, tiles
    of 8 lines: 3 x 18 = 54 lines leave a ragged last tile."""
    nx, ny, nz = 512, 3, 18
    faces = W.tanh_faces(ny, 1.6)
    g = oracle.Grid(nx, nz, faces)
    f = oracle.divergence(g, *W.random_velocity(5, nx, ny, nz))
    want = oracle.solve(g, f)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32_REFINED, pdd_parts=1, fp64_low_modes=4, refine_steps=2,
                  device=DEV)
    got = plan.solve(to_dev(f))
    torch.cuda.synchronize()
    assert relerr(got.cpu().numpy(), want) <= 1e-12
    assert plan.device_status() == 0


@pytest.mark.parametrize("nx,ny,nz,steps", [(768, 5, 9, 1), (768, 4, 6, 2), (1024, 3, 6, 2), (2048, 5, 3, 1)])
def test_fp32_refined_solve_register_residual_lengths(P, nx, ny, nz, steps):
    """The residual pass with the register transform at Nx/2 = 384 (240 threads: a partial last
    warp skips the residual phase; tiles of 10 lines), 512 and 1024, every line count leaving a
    ragged last tile; one correction at the one-correction bound, two at the FP64 bar."""
    faces = W.tanh_faces(ny, 1.7)
    g = oracle.Grid(nx, nz, faces)
    f = oracle.divergence(g, *W.random_velocity(7, nx, ny, nz))
    want = oracle.solve(g, f)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32_REFINED, pdd_parts=1, fp64_low_modes=4,
                  refine_steps=steps, device=DEV)
    got = plan.solve(to_dev(f))
    torch.cuda.synchronize()
    assert relerr(got.cpu().numpy(), want) <= (2e-9 if steps == 1 else 1e-12)
    assert plan.device_status() == 0


@pytest.mark.parametrize("steps", [2, 3])
def test_fp32_refined_solve_generic_fft(P, steps):
    """The refined solve through the runtime-generic kernels (POISSON_GENERIC_FFT; Nx/2 = 18 has
    no specialised transform either): their residual producer forms the first correction's
    residual from f and stores it, and the later ones from that stored residual."""
    nx, ny, nz = 36, 12, 18
    faces = W.tanh_faces(ny, 2.0)
    g = oracle.Grid(nx, nz, faces)
    f = oracle.divergence(g, *W.random_velocity(8, nx, ny, nz))
    want = oracle.solve(g, f)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32_REFINED, pdd_parts=1, fp64_low_modes=4,
                  refine_steps=steps, flags=P.POISSON_GENERIC_FFT, device=DEV)
    got = plan.solve(to_dev(f))
    torch.cuda.synchronize()
    assert relerr(got.cpu().numpy(), want) <= 1e-12


def test_bounded_wait_runs_out_and_reports_timeout(P):
    """POISSON_SELFTEST_WAIT makes the bulk-copy-staged x-transform skip its first copy: its
    bounded mbarrier wait gives up (~2 s), the device status reads PS_ETIMEOUT, and the context
    stays usable for the next solve."""
    from paper_2104_08863_gb300 import _native
    nx, ny, nz = 512, 4, 16
    faces = W.tanh_faces(ny, 1.5)
    f = np.random.default_rng(9).standard_normal((ny, nz, nx))
    bad = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32_REFINED, pdd_parts=1, flags=P.POISSON_SELFTEST_WAIT,
                 device=DEV)
    bad.solve(to_dev(f))
    torch.cuda.synchronize()
    assert bad.device_status() == _native.PS_ETIMEOUT
    g = oracle.Grid(nx, nz, faces)
    f -= np.einsum("j,jki->", g.dy, f) / (g.dy.sum() * nx * nz)
    good = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32_REFINED, pdd_parts=1, refine_steps=2, device=DEV)
    got = good.solve(to_dev(f))
    torch.cuda.synchronize()
    assert good.device_status() == 0
    assert relerr(got.cpu().numpy(), oracle.solve(g, f)) <= 1e-12


@pytest.mark.parametrize("prec,steps,tol", [(0, 1, 1e-12), (1, 1, 2e-5), (2, 2, 1e-12)])
def test_solve_adjoint_matches_oracle_transpose(P, prec, steps, tol):
    """poisson_solve_adjoint = S^T (the transpose of the gauged solve) against the oracle's
    solve_transposed, itself pinned to the dense transpose of the oracle's solve."""
    nx, ny, nz = 48, 24, 32
    faces = W.tanh_faces(ny, 1.9)
    g = oracle.Grid(nx, nz, faces)
    r = np.random.default_rng(12).standard_normal((ny, nz, nx))
    want = oracle.solve_transposed(g, r)
    dtype = torch.float32 if prec == P.PP_FP32 else torch.float64
    plan = P.Plan(nx, ny, nz, faces, precision=prec, pdd_parts=4, fp64_low_modes=4, refine_steps=steps, device=DEV)
    rt = to_dev(r, dtype)
    got = plan.solve_adjoint(rt)
    torch.cuda.synchronize()
    assert relerr(got.double().cpu().numpy(), want) <= tol
    same = rt.clone()
    plan.solve_adjoint(same, out=same)   # in place
    torch.cuda.synchronize()
    assert relerr(same.double().cpu().numpy(), want) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32", "refined"])
def test_host_projection_equals_device_projection(P, prec):
    """projection_step_host (pinned host buffers in, results copied back) equals projection_step
    on device buffers: bit for bit, except the refined form's pressure gauge (FP64 atomics)."""
    nx, ny, nz = 48, 20, 24
    faces = W.tanh_faces(ny, 1.7)
    case = W.ChannelCase("h", nx, ny, nz, 1.7)
    u, v, w = W.poiseuille_plus_noise(4, case)
    precision = {"fp64": P.PP_FP64, "fp32": P.PP_FP32, "refined": P.PP_FP32_REFINED}[prec]
    dtype = torch.float32 if prec == "fp32" else torch.float64
    plan = P.Plan(nx, ny, nz, faces, precision=precision, refine_steps=2 if prec == "refined" else 1, device=DEV)
    ut, vt, wt = (to_dev(a).to(dtype) for a in (u, v, w))
    pt = torch.empty(ny, nz, nx, dtype=dtype, device=DEV)
    plan.project(ut, vt, wt, 1e-3, p_out=pt)
    hosts = [torch.from_numpy(np.ascontiguousarray(a)).to(dtype).pin_memory() for a in (u, v, w)]
    ph = torch.empty(ny, nz, nx, dtype=dtype).pin_memory()
    staging = (torch.empty_like(ut), torch.empty_like(vt), torch.empty_like(wt), torch.empty_like(pt))
    plan.project_host(*hosts, 1e-3, staging, p_h=ph)
    torch.cuda.synchronize()
    for q, (dev_t, host_t) in enumerate(zip((ut, vt, wt, pt), (*hosts, ph))):
        if prec == "refined":
            d = float((dev_t.cpu() - host_t).abs().max() / host_t.abs().max())
            assert d <= (1e-13 if q < 3 else 1e-10), (q, d)
        else:
            assert torch.equal(dev_t.cpu(), host_t)


def test_fp64_fma_rate_is_measured_and_checks_its_scratch(P):
    """poisson_fp64_fma_rate: a positive FP64 FMA throughput no larger than two FMAs per clock per
    SM at the highest SM clock (the GB300 rate), and PS_EINVAL for a scratch buffer too small."""
    import ctypes
    from paper_2104_08863_gb300 import _native
    rate = P.fp64_fma_rate(DEV)
    props = torch.cuda.get_device_properties(DEV)
    assert 0.0 < rate <= 2 * 2 * props.multi_processor_count * 2.2   # GFLOP/s, 2.2 GHz bound
    small = torch.empty(64, dtype=torch.uint8, device=DEV)
    out = ctypes.c_double()
    st = _native.lib().poisson_fp64_fma_rate(small.data_ptr(), small.numel(), None, ctypes.byref(out))
    assert st != 0
