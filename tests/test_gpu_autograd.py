"""The projection inside torch.autograd.Function with its hand-written adjoint backward.

Workload: FP32 projection on the 256 x 192 x 256 channel (tanh 1.8), velocity seed 3 N(0,1)
per component, loss sum(w . u) with seed-4 U(-1, 1) weights.  The backward (P^T w through the
same FFT/PDD kernels) is checked against
* central finite differences with h = 1e-3 computed with the FP64 projection, on 64 seed-6
  N(0,1) directions (the map is linear, so the difference quotient is exact up to rounding):
  agreement ~1e-5 relative for the FP32 backward;
* the oracle's FP64 gradient P^T w, elementwise.
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


def test_projection_autograd_fp32_vs_finite_differences_and_oracle(P):
    case = W.CHANNEL_256
    nx, ny, nz = case.nx, case.ny, case.nz
    faces = W.tanh_faces(ny, case.stretch)
    dt = 1e-3
    plan32 = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32, device=DEV)
    plan64 = P.Plan(nx, ny, nz, faces, precision=P.PP_FP64, device=DEV)
    u0 = [torch.from_numpy(a).to(DEV) for a in W.random_velocity(3, nx, ny, nz)]
    wts = [torch.from_numpy(a).to(DEV) for a in W.weight_field(4, nx, ny, nz)]
    x = [a.float().requires_grad_(True) for a in u0]
    out = P.ProjectionFn.apply(x[0], x[1], x[2], plan32, dt)
    loss = sum((o.double() * wt).sum() for o, wt in zip(out, wts))
    loss.backward()
    grad = [a.grad.double() for a in x]

    def J(vel):
        a, b, c = (t.clone() for t in vel)
        plan64.project(a, b, c, dt)
        return sum(float((o * wt).sum()) for o, wt in zip((a, b, c), wts))

    rng = np.random.default_rng(6)
    h = 1e-3
    errs = []
    for _ in range(64):
        d = [torch.from_numpy(rng.standard_normal(tuple(t.shape))).to(DEV) for t in u0]
        fd = (J([a + h * e for a, e in zip(u0, d)]) - J([a - h * e for a, e in zip(u0, d)])) / (2 * h)
        an = sum(float((gr * e).sum()) for gr, e in zip(grad, d))
        scale = sum(float((gr.abs() * e.abs()).sum()) for gr, e in zip(grad, d))
        errs.append(abs(fd - an) / scale)
    assert max(errs) <= 2e-5, max(errs)
    g = oracle.Grid(nx, nz, faces)
    want = oracle.project_adjoint(g, *(t.cpu().numpy() for t in wts))
    for got, ref in zip(grad, want):
        assert np.max(np.abs(got.cpu().numpy() - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_gradcheck_fp64_tiny(P):
    nx, ny, nz = 8, 6, 4
    plan = P.Plan(nx, ny, nz, W.tanh_faces(ny, 1.4), precision=P.PP_FP64, pdd_parts=2, device=DEV)
    rng = np.random.default_rng(7)
    x = [torch.from_numpy(rng.standard_normal(s)).to(DEV).requires_grad_(True)
         for s in ((ny, nz, nx), (ny + 1, nz, nx), (ny, nz, nx))]
    fn = lambda a, b, c: P.ProjectionFn.apply(a, b, c, plan, 0.5)
    assert torch.autograd.gradcheck(fn, tuple(x), eps=1e-6, atol=1e-8, rtol=1e-6)
