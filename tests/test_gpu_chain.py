"""The kx-slab chain of the FP32 spectral middle (poisson_plan_set_chain): the forward
z-transform, the wall-normal PDD solves and the inverse z-transform run slab by slab (one or two
streams).  Every column is computed by the same kernels as in the whole-spectrum order, so FP32
results are bit-identical to it; the refined form's gauge accumulates the pressure's weighted sum
with atomic additions (order-dependent rounding): 1e-13.  Both are also checked against the
oracle at the tolerances of the FP32 forms."""
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


def _rhs(nx, ny, nz, faces, seed):
    g = oracle.Grid(nx, nz, faces)
    f = oracle.divergence(g, *W.random_velocity(seed, nx, ny, nz))
    return g, f


@pytest.mark.parametrize("streams", [1, 2])
def test_fp32_chain_bit_identical_and_matches_oracle(P, streams):
    # 49 spectral columns in slabs of 32 (a ragged last slab), 16 PDD blocks of 6 rows
    nx, ny, nz = 96, 96, 64
    faces = W.tanh_faces(ny, 2.0)
    g, f = _rhs(nx, ny, nz, faces, 11)
    f -= np.einsum("j,jki->", g.dy, f) / (g.dy.sum() * nx * nz)
    want = oracle.solve(g, f)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32, pdd_parts=16, fp64_low_modes=4, device=DEV)
    ft = torch.from_numpy(f).to(DEV, torch.float32)
    ref = plan.solve(ft).clone()
    plan.set_chain(32, streams)
    for _ in range(2):
        got = plan.solve(ft)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
    assert relerr(got.double().cpu().numpy(), want) <= 2e-5
    plan.set_chain(0)
    assert torch.equal(plan.solve(ft), ref)


@pytest.mark.parametrize("streams", [1, 2])
def test_refined_chain_matches_whole_order_and_oracle(P, streams):
    # 65 spectral columns in slabs of 16 (z tile 16 at nz = 512, 8 systems per PDD CTA at P = 32)
    nx, ny, nz = 128, 64, 512
    faces = W.tanh_faces(ny, 2.2)
    g, f = _rhs(nx, ny, nz, faces, 12)
    want = oracle.solve(g, f)
    plan = P.Plan(nx, ny, nz, faces, precision=P.PP_FP32_REFINED, pdd_parts=32, fp64_low_modes=4,
                  refine_steps=1, device=DEV)
    ft = torch.from_numpy(f).to(DEV)
    ref = plan.solve(ft).clone()
    plan.set_chain(16, streams)
    got = plan.solve(ft)
    torch.cuda.synchronize()
    assert float((got - ref).abs().max() / ref.abs().max()) <= 1e-13
    assert relerr(got.cpu().numpy(), want) <= 2e-9
    assert plan.device_status() == 0


def test_chain_refuses_fp64_plans(P):
    from paper_2104_08863_gb300 import _native
    plan = P.Plan(64, 32, 64, W.tanh_faces(32, 1.5), precision=P.PP_FP64, pdd_parts=4, device=DEV)
    with pytest.raises(_native.PoissonError):
        plan.set_chain(32, 1)
