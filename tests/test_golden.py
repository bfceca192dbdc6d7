"""Golden fixtures (tests/golden/, written by make_golden.py from the oracle): the oracle still
reproduces them on the CPU, and the CUDA path matches them on the GPU."""
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASE = W.CHANNEL_32


def _load(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, f"channel32_{name}_pressure.txt")) if not l.startswith("#")]
    return [(int(j), int(k), int(i), float(v)) for j, k, i, v in rows]


def _rhs(name):
    faces = W.tanh_faces(CASE.ny, CASE.stretch)
    g = oracle.Grid(CASE.nx, CASE.nz, faces)
    if name == "manufactured":
        return g, faces, W.manufactured_rhs(CASE.nx, CASE.ny, CASE.nz, faces)
    return g, faces, oracle.divergence(g, *W.random_velocity(0, CASE.nx, CASE.ny, CASE.nz))


@pytest.mark.parametrize("name", ["manufactured", "random_divergence"])
def test_oracle_reproduces_golden(name):
    g, _, f = _rhs(name)
    p = oracle.solve(g, f)
    for j, k, i, v in _load(name):
        assert abs(p[j, k, i] - v) <= 1e-13 * max(1.0, abs(v))


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["manufactured", "random_divergence"])
def test_cuda_path_matches_golden(name):
    import torch
    from paper_2104_08863_gb300 import build as b
    b.build()
    import paper_2104_08863_gb300 as P
    g, faces, f = _rhs(name)
    plan = P.Plan(CASE.nx, CASE.ny, CASE.nz, faces, precision=P.PP_FP64, tridiag=P.PT_THOMAS,
                  device=torch.device("cuda:0"))
    p = plan.solve(torch.from_numpy(f).to("cuda:0")).cpu().numpy()
    gold = _load(name)
    scale = max(abs(v) for *_, v in gold)
    for j, k, i, v in gold:
        assert abs(p[j, k, i] - v) <= 1e-12 * scale


GOLDEN_1536 = os.path.join(GOLDEN, "channel1536_seed2_modes.json")


def test_golden_1536_modes_solve_their_wall_normal_systems():
    """The stored sampled-mode solutions of the 1536x768x1024 channel (make_golden_1536.py) satisfy
    their tridiagonal systems of Eq. 9, row by row, with the stored mode rhs: a residual check that
    is independent of the Thomas recurrence that produced them."""
    import json
    d = json.load(open(GOLDEN_1536))
    nx, ny, nz = d["grid"]
    g = oracle.Grid(nx, nz, W.tanh_faces(ny, d["stretch"]), d["lx"], d["lz"])
    a, c = g.lower, g.upper
    lamx, lamz = g.lambda_x(), g.lambda_z()
    assert len(d["modes"]) >= 6
    for m in d["modes"]:
        F = np.array([complex(re, im) for re, im in m["F"]])
        Pm = np.array([complex(re, im) for re, im in m["P"]])
        assert F.shape == Pm.shape == (ny,)
        diag = -(a + c) + lamx[m["kx"]] + lamz[m["kz"]]
        r = diag * Pm - F
        r[1:] += a[1:] * Pm[:-1]
        r[:-1] += c[:-1] * Pm[1:]
        assert np.max(np.abs(r)) <= 1e-12 * np.max(np.abs(F)), (m["kx"], m["kz"])
