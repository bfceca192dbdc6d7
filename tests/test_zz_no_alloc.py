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


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
def test_static_workspace_matches_poisson_solve_twice(P, precision, tol):
    dev = torch.device("cuda:0")
    nx, ny, nz = 48, 32, 24
    plan = P.Plan(nx, ny, nz, W.tanh_faces(ny, 1.8), precision=precision, pdd_parts=4, device=dev)
    assert plan.workspace_bytes <= P._native.POISSON_STATIC_WS_MAX_BYTES
    dtype = plan.dtype
    f = torch.from_numpy(W.random_field(31, (ny, nz, nx))).to(device=dev, dtype=dtype)
    ref = plan.solve(f)
    torch.cuda.synchronize()
    for _ in range(2):
        got = _static_solve(plan, f)
        assert _relerr(got, ref) <= tol


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
