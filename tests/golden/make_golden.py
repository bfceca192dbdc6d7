"""Writes the golden fixtures of this directory from the CPU oracle only.

The paper prints no worked numerical example, so the fixtures are oracle outputs on the
32x32x32 channel (tanh 1.5) at sampled cells, kept as a regression anchor: the CPU tests check
that the oracle still reproduces them, the GPU tests compare the CUDA path with them.
Run: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402

SAMPLES = [(0, 0, 0), (0, 5, 31), (1, 16, 3), (7, 9, 20), (15, 31, 0), (16, 2, 17), (30, 12, 8), (31, 31, 31)]


def main():
    case = W.CHANNEL_32
    faces = W.tanh_faces(case.ny, case.stretch)
    g = oracle.Grid(case.nx, case.nz, faces)
    rhs = {"manufactured": W.manufactured_rhs(case.nx, case.ny, case.nz, faces),
           "random_divergence": oracle.divergence(g, *W.random_velocity(0, case.nx, case.ny, case.nz))}
    for name, f in rhs.items():
        p = oracle.solve(g, f)
        path = os.path.join(HERE, f"channel32_{name}_pressure.txt")
        with open(path, "w") as fh:
            fh.write(f"# oracle.solve on the 32x32x32 channel (tanh 1.5), rhs: {name}; j k i p[j,k,i] (repr)\n")
            for j, k, i in SAMPLES:
                fh.write(f"{j} {k} {i} {float(p[j, k, i])!r}\n")


if __name__ == "__main__":
    main()
