"""Independent FP64 CPU oracle for the staggered-channel pressure-Poisson projection.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The GPU library never calls it and shares no
code, table or constant generator with it.

What it computes (Sec. 2 of the paper, Eqs. 3-9, with the readings listed below):

* ``grid``      -- metrics of the stretched wall-normal grid and the modified wavenumbers
                   of the periodic three-point stencils (Eq. 9's eigenvalues).
* ``stencils``  -- the staggered finite-volume divergence D, gradient G, Laplacian
                   L_h = D G (Eq. 8 generalised to the stretched y grid) and their transposes.
* ``tridiag``   -- the textbook Thomas algorithm (Sec. 2.1) in extended precision, and the
                   PDD algorithm of Sec. 2.2 (Eqs. 11-21, five-step procedure) with either the
                   exact reduced system Z of Eq. 21 or its truncated 2x2 form.
* ``poisson``   -- the pressure solve L_h p = f - mean(f) with a zero volume-weighted mean
                   gauge, the projection u = u* - dt G p (Eqs. 4 and 7) and its adjoint.
* ``momentum``  -- the momentum right-hand side -N(u) + nu lap(u) + F (central, divergence
                   form, no-slip walls), Heun's RK2 predictor (Eqs. 5-6) and one full timestep.

Readings of the paper (the text is silent or garbled on these points):

* axes: x streamwise, y wall-normal (stretched), z spanwise, as in Sec. 5;
* Eq. 9's centre coefficient is -2 (the printed +2 is a sign slip);
* the pressure boundary condition is homogeneous Neumann (zero flux through the walls);
* the transforms in x and z are complex-exponential DFTs (periodic directions);
* cell centres in y are midpoints of the adjacent faces;
* the singular (kx, kz) = (0, 0) mode is made compatible by removing the volume-weighted
  mean of f and is gauged by a zero volume-weighted mean of p;
* steps (6) and (8) of Sec. 3.2 are inverse transforms;
* advection is the divergence form with arithmetic two-point face averages, the no-slip wall
  enters the diffusion through the wall value 0 half a cell from the first node, and the flow is
  driven by a constant streamwise body force.

Parity status per function: every public function here is pinned by the ``-m "not gpu"``
tests in ``tests/test_oracle_pins.py`` (closed forms, dense LU, convergence order,
brute-force transposes and invariants) and ``tests/test_oracle_momentum.py`` (closed forms of
the staggered differences, conservation, self-adjoint diffusion, Heun vs its Taylor polynomial).
"""
from .grid import Grid
from .stencils import divergence, gradient, laplacian, divergence_T, gradient_T
from .tridiag import thomas, pdd
from .poisson import solve, solve_pdd, solve_transposed, project, project_adjoint, residual
from .momentum import momentum_rhs, rk2_predictor, timestep

__all__ = [
    "Grid", "divergence", "gradient", "laplacian", "divergence_T", "gradient_T",
    "thomas", "pdd", "solve", "solve_pdd", "solve_transposed", "project", "project_adjoint", "residual",
    "momentum_rhs", "rk2_predictor", "timestep",
]
