"""Batched uneven-size solves in one graph launch, and the autotuner.

Workload: 64 instances drawn with default_rng(5) (Nx, Nz from {64..384}, Ny from {48..192},
tanh stretching U(1, 2.5)); each rhs the divergence of a seeded N(0,1) velocity, FP32.
Every batched result must equal the same plan solved alone (same kernels: bit-identical up to
the order of concurrent work, which does not change any arithmetic), and the smallest
instances are checked against the oracle at the FP32 tolerance.
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


def test_batched_64_uneven_instances_match_single_solves_and_oracle(P):
    cases = W.batch_instances(5, 64)
    specs = [dict(nx=c.nx, ny=c.ny, nz=c.nz, y_faces=W.tanh_faces(c.ny, c.stretch)) for c in cases]
    bp = P.BatchPlan(specs, precision=P.PP_FP32, device=DEV)
    rng = np.random.default_rng(55)
    rhs = [torch.from_numpy(rng.standard_normal((c.ny, c.nz, c.nx))).float().to(DEV) for c in cases]
    outs = bp.solve(rhs)
    outs2 = bp.solve(rhs)          # replays the captured graph
    torch.cuda.synchronize()
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)
    order = np.argsort([c.npoints for c in cases])
    for idx in list(order[:6]) + list(order[-2:]):
        c = cases[idx]
        single = P.Plan(c.nx, c.ny, c.nz, specs[idx]["y_faces"], precision=P.PP_FP32, device=DEV)
        ref = single.solve(rhs[idx])
        torch.cuda.synchronize()
        assert torch.allclose(outs[idx], ref, rtol=0, atol=1e-6 * float(ref.abs().max()))
    for idx in order[:4]:
        c = cases[idx]
        g = oracle.Grid(c.nx, c.nz, specs[idx]["y_faces"])
        want = oracle.solve(g, rhs[idx].double().cpu().numpy())
        got = outs[idx].double().cpu().numpy()
        assert np.max(np.abs(got - want)) <= 2e-5 * np.max(np.abs(want))


def test_persistent_launch_matches_graph_branches(P):
    """The persistent work-queue launch and the graph of per-instance branches give the same
    results (the same tile arithmetic; the low modes by FP64 Thomas instead of FP64 PDD)."""
    cases = W.batch_instances(5, 24)
    specs = [dict(nx=c.nx, ny=c.ny, nz=c.nz, y_faces=W.tanh_faces(c.ny, c.stretch)) for c in cases]
    rng = np.random.default_rng(56)
    rhs = [torch.from_numpy(rng.standard_normal((c.ny, c.nz, c.nx))).float().to(DEV) for c in cases]
    pers = P.BatchPlan(specs, precision=P.PP_FP32, device=DEV, persistent=True)
    outs = pers.solve(rhs)
    assert pers.last_launch_count == 1          # one persistent kernel per graph launch
    branch = P.BatchPlan(specs, precision=P.PP_FP32, device=DEV)
    refs = branch.solve(rhs)
    assert branch.last_launch_count > len(cases)
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.allclose(o, r, rtol=0, atol=1e-6 * float(r.abs().max()))
    assert pers.device_status() == 0
    # a second pointer set re-captures the graph
    outs2 = [torch.empty_like(r) for r in rhs]
    pers.solve(rhs, out=outs2)
    torch.cuda.synchronize()
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)


def test_persistent_bounded_wait_runs_out_and_reports_timeout(P):
    """POISSON_SELFTEST_WAIT: the first x-tile of instance 0 is never counted done, so the waits of its
    next pass run out (about a second), the launch aborts and the batch status reads PS_ETIMEOUT; the
    context stays usable and a normal batch solves correctly afterwards."""
    from paper_2104_08863_gb300 import _native
    specs = [dict(nx=64, ny=48, nz=64, y_faces=W.tanh_faces(48, 1.5)),
             dict(nx=96, ny=64, nz=96, y_faces=W.tanh_faces(64, 2.0))]
    rng = np.random.default_rng(57)
    rhs = [torch.from_numpy(rng.standard_normal((s["ny"], s["nz"], s["nx"]))).float().to(DEV) for s in specs]
    bad = P.BatchPlan(specs, precision=P.PP_FP32, device=DEV, persistent=True, selftest_wait=True)
    bad.solve(rhs)
    torch.cuda.synchronize()
    assert bad.last_launch_count == 1
    assert bad.device_status() == _native.PS_ETIMEOUT
    good = P.BatchPlan(specs, precision=P.PP_FP32, device=DEV, persistent=True)
    outs = good.solve(rhs)
    torch.cuda.synchronize()
    assert good.device_status() == 0
    for s, r, o in zip(specs, rhs, outs):
        g = oracle.Grid(s["nx"], s["nz"], s["y_faces"])
        want = oracle.solve(g, r.double().cpu().numpy())
        assert np.max(np.abs(o.double().cpu().numpy() - want)) <= 2e-5 * np.max(np.abs(want))


def test_batched_mixed_precisions_and_bad_pointers(P):
    specs = [dict(nx=32, ny=16, nz=24, y_faces=W.tanh_faces(16, 1.5), pdd_parts=2),
             dict(nx=48, ny=24, nz=16, y_faces=W.tanh_faces(24, 2.0), pdd_parts=3)]
    bp = P.BatchPlan(specs, precision=P.PP_FP64, device=DEV)
    rng = np.random.default_rng(9)
    rhs = [torch.from_numpy(rng.standard_normal((s["ny"], s["nz"], s["nx"]))).to(DEV) for s in specs]
    outs = bp.solve(rhs)
    torch.cuda.synchronize()
    for s, r, o in zip(specs, rhs, outs):
        g = oracle.Grid(s["nx"], s["nz"], s["y_faces"])
        want = oracle.solve(g, r.cpu().numpy())
        assert np.max(np.abs(o.cpu().numpy() - want)) <= 1e-12 * np.max(np.abs(want))
    with pytest.raises(ValueError):
        bp.solve(rhs[:1])


def test_autotune_returns_a_valid_configuration(P):
    faces = W.tanh_faces(96, 2.0)
    parts, flags, ms = P.autotune(128, 96, 64, faces, precision=P.PP_FP32)
    assert parts == 1 or (96 % parts == 0 and 96 // parts >= 4)
    assert flags in (0, P.POISSON_GENERIC_FFT)
    assert ms > 0
    plan = P.Plan(128, 96, 64, faces, precision=P.PP_FP32, tridiag=P.PT_THOMAS if parts == 1 else P.PT_PDD_EXACT,
                  pdd_parts=parts, flags=flags, device=DEV)
    g = oracle.Grid(128, 64, faces)
    f = W.random_field(12, (96, 64, 128))
    got = plan.solve(torch.from_numpy(f).float().to(DEV)).double().cpu().numpy()
    want = oracle.solve(g, f)
    assert np.max(np.abs(got - want)) <= 2e-5 * np.max(np.abs(want))
