"""poisson_solve_static_ws: the solve for callers that cannot allocate device memory.

It must give the same result as poisson_solve (caller workspace) on the same plan, call
after call, although every call reuses one library-owned device array.  This file is named
to be collected last, so a run that stops at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2104_08863_gb300 import build as b
    b.build()
    import paper_2104_08863_gb300 as mod
    return mod


def _static_solve(plan, rhs):
    from paper_2104_08863_gb300 import _native
    out = torch.full_like(rhs, float("nan"))
    rc = _native.lib().poisson_solve_static_ws(plan._h, rhs.data_ptr(), out.data_ptr(),
                                                torch.cuda.current_stream().cuda_stream)
    assert rc == _native.PS_OK, _native.status_string(rc)
    torch.cuda.synchronize()
    return out


def _relerr(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# PP_FP64 and PP_FP32 run the same deterministic kernels on the same tables in both entry points,
# so their results agree bit for bit; the refined form accumulates the pressure's weighted sum
# with atomic additions (order-dependent rounding of the gauge constant): 1e-12.
@pytest.mark.parametrize("precision,tol", [(0, 0.0), (1, 0.0), (2, 1e-12)])
def test_static_workspace_matches_poisson_solve_twice(P, precision, tol):
    dev = torch.device("cuda:0")
    nx, ny, nz = 48, 32, 24
    plan = P.Plan(nx, ny, nz, W.tanh_faces(ny, 1.8), precision=precision, pdd_parts=4, refine_steps=2,
                  device=dev)
    assert plan.workspace_bytes <= P._native.POISSON_STATIC_WS_MAX_BYTES
    dtype = plan.dtype
    f = torch.from_numpy(W.random_field(31, (ny, nz, nx))).to(device=dev, dtype=dtype)
    ref = plan.solve(f)
    torch.cuda.synchronize()
    for _ in range(2):
        got = _static_solve(plan, f)
        assert _relerr(got, ref) <= tol
    if precision == 2:   # the refined solve re-reads its right-hand side: no in-place call
        from paper_2104_08863_gb300 import _native
        rc = _native.lib().poisson_solve_static_ws(plan._h, f.data_ptr(), f.data_ptr(),
                                                    torch.cuda.current_stream().cuda_stream)
        assert rc == _native.PS_EINVAL


def test_static_workspace_alternating_precisions(P):
    """Plans of different precision (and table layouts) take turns on the one array."""
    dev = torch.device("cuda:0")
    nx, ny, nz = 48, 24, 36
    faces = W.tanh_faces(ny, 2.0)
    plans = [P.Plan(nx, ny, nz, faces, precision=prec, pdd_parts=parts, refine_steps=1, device=dev)
             for prec, parts in ((2, 4), (0, 3), (1, 6))]
    f64 = torch.from_numpy(W.random_field(34, (ny, nz, nx))).to(dev)
    rhs = [f64, f64, f64.float()]
    refs = [pl.solve(r) for pl, r in zip(plans, rhs)]
    torch.cuda.synchronize()
    for _ in range(2):
        for pl, r, ref, tol in zip(plans, rhs, refs, (1e-12, 0.0, 0.0)):
            assert _relerr(_static_solve(pl, r), ref) <= tol


def test_static_workspace_rejects_batched_plans(P):
    from paper_2104_08863_gb300 import _native
    dev = torch.device("cuda:0")
    spec = dict(nx=16, ny=8, nz=8, y_faces=W.tanh_faces(8, 1.5))
    bp = P.BatchPlan([spec, spec], precision=P.PP_FP32, device=dev)
    x = torch.zeros(8, 8, 16, dtype=torch.float32, device=dev)
    rc = _native.lib().poisson_solve_static_ws(bp._h, x.data_ptr(), x.data_ptr(),
                                                torch.cuda.current_stream().cuda_stream)
    assert rc == _native.PS_EINVAL


def test_static_workspace_alternating_plans_and_size_limit(P):
    dev = torch.device("cuda:0")
    a = P.Plan(32, 32, 32, W.tanh_faces(32, 1.5), precision=0, pdd_parts=2, device=dev)
    b = P.Plan(24, 16, 36, W.tanh_faces(16, 2.0), precision=0, pdd_parts=1, device=dev)
    fa = torch.from_numpy(W.random_field(32, (32, 32, 32))).to(dev)
    fb = torch.from_numpy(W.random_field(33, (16, 36, 24))).to(dev)
    ra, rb = a.solve(fa), b.solve(fb)
    for _ in range(2):
        assert _relerr(_static_solve(a, fa), ra) <= 1e-12
        assert _relerr(_static_solve(b, fb), rb) <= 1e-12
    from paper_2104_08863_gb300 import _native
    big = P.Plan(256, 64, 256, W.tanh_faces(64, 1.5), precision=0, device=dev)
    assert big.workspace_bytes > _native.POISSON_STATIC_WS_MAX_BYTES
    x = torch.zeros(64, 256, 256, dtype=torch.float64, device=dev)
    rc = _native.lib().poisson_solve_static_ws(big._h, x.data_ptr(), x.data_ptr(),
                                                torch.cuda.current_stream().cuda_stream)
    assert rc == _native.PS_EUNSUPPORTED
