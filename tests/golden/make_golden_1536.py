"""Writes channel1536_seed2_modes.json from the CPU oracle only: the exact wall-normal solutions
of sampled (kx, kz) modes of the 1536x768x1024 channel (tanh 2.2) for the right-hand side
f = D(u, v, w), (u, v, w) the seed-2 N(0, 1) staggered velocity (workloads.random_velocity).

For each mode the script stores F_j = sum_{k,i} f[j,k,i] e^{-2 pi i (kz k / Nz + kx i / Nx)} (the
complex DFT of Eq. 9 by direct summation, for every wall-normal row j) and the solution P_j of
the mode's tridiagonal system of Eq. 9 (oracle Thomas in extended precision).  The volume-weighted
mean that the solve removes only touches the (0, 0) mode, which is not sampled.  The modes are the
weakest ones (the FP64 low-mode set |kx|, |kz| <= 4 and its first FP32 neighbours), a middle and
the highest.  The GPU tests and bench.py compare the DFT of their pressure at these modes with P.

Needs about 40 GB of host memory.  Run: python tests/golden/make_golden_1536.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from oracle.tridiag import thomas  # noqa: E402

MODES = [(1, 0), (0, 1), (4, 4), (5, 1), (0, 5), (3, 1020), (300, 700), (768, 512)]
OUT = os.path.join(HERE, "channel1536_seed2_modes.json")


def rhs_seed2(case):
    """f = D(u, v, w) of the seed-2 velocity, computed one wall-normal plane at a time."""
    faces = W.tanh_faces(case.ny, case.stretch)
    u, v, w = W.random_velocity(2, case.nx, case.ny, case.nz)
    f = np.empty((case.ny, case.nz, case.nx))
    for j in range(case.ny):
        gj = oracle.Grid(case.nx, case.nz, faces[j:j + 2], case.lx, case.lz)
        f[j] = oracle.divergence(gj, u[j:j + 1], v[j:j + 2], w[j:j + 1])[0]
    return f


def main():
    case = W.CHANNEL_1536
    faces = W.tanh_faces(case.ny, case.stretch)
    g = oracle.Grid(case.nx, case.nz, faces, case.lx, case.lz)
    t0 = time.time()
    f = rhs_seed2(case)
    print(f"rhs built in {time.time() - t0:.0f} s", flush=True)
    a, c = g.lower, g.upper
    lamx, lamz = g.lambda_x(), g.lambda_z()
    out = {"grid": [case.nx, case.ny, case.nz], "stretch": case.stretch, "lx": case.lx, "lz": case.lz,
           "rhs": "D(u, v, w), (u, v, w) = workloads.random_velocity(2, 1536, 768, 1024)",
           "max_abs_f": float(np.max(np.abs(f))), "modes": []}
    for kx, kz in MODES:
        ex = np.exp(-2j * np.pi * kx * np.arange(case.nx) / case.nx)
        ez = np.exp(-2j * np.pi * kz * np.arange(case.nz) / case.nz)
        F = np.einsum("jki,k,i->j", f, ez, ex, optimize=True)
        P = thomas(a, -(a + c) + lamx[kx] + lamz[kz], c, F)
        out["modes"].append({"kx": kx, "kz": kz,
                             "F": [[float(z.real), float(z.imag)] for z in F],
                             "P": [[float(z.real), float(z.imag)] for z in P]})
        print(f"mode ({kx}, {kz}) done at {time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=0)


if __name__ == "__main__":
    main()
