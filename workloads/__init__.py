"""Seeded synthetic inputs for the low-memory S_N-DG transport problem (Sun & Hauck, arXiv 1907.01027).

This module builds problem *data* only: angular quadrature tables, uniform Cartesian meshes, per-cell
cross sections, sources given as Q1 Legendre coefficients, and inflow boundary data.  It contains none of
the discretisation's arithmetic (no DG forms, no sweeps, no reductions), so both the FP64 oracle and the
CUDA path may take their inputs from here.

Conventions shared by every consumer (they define the inputs, not the method):

* Mesh: ``n x n`` square cells of side ``h`` on ``[x0, x0 + n h] x [y0, y0 + n h]``; cell ``(i, j)`` (``i``
  along x, ``j`` along y) has linear index ``p = j * n + i`` and centre ``(x0 + (i + 1/2) h, y0 + (j + 1/2) h)``.
* Cell basis (Legendre, orthogonal, constant first as Section 3.2 requires): ``b0 = 1, b1 = xi, b2 = eta,
  b3 = xi * eta`` with ``xi = 2 (x - x_c) / h`` and ``eta = 2 (y - y_c) / h``.
* Sources are Legendre coefficients of ``q`` on each cell: layout 1 is ``[n_x][4]`` (isotropic), layout 2 is
  ``[n_Omega][n_x][4]`` (angle dependent, used by manufactured solutions, Section 4.1 notes ``q`` may depend
  on angle).
* Inflow data ``alpha`` (eq-main boundary condition) is given per angle, per side and per boundary face as
  the two Legendre coefficients ``(a0, a1)`` of its linear projection along the face:
  ``alpha(t) = a0 + a1 t`` with ``t`` in [-1, 1] increasing with the global coordinate along the face.
  Layout ``[n_Omega][4][n][2]`` with sides ``0 = west (x = x0), 1 = east, 2 = south (y = y0), 3 = north``.
"""
from .quadrature import level_symmetric_2d, quadrant_of
from .problems import (Problem, uniform_problem, config1, config2, config3, config4, config5,
                       mms_problem, diffusion_limit_problem, legendre_project_cell, legendre_project_face)

__all__ = ["level_symmetric_2d", "quadrant_of", "Problem", "uniform_problem", "config1", "config2",
           "config3", "config4", "config5", "mms_problem", "diffusion_limit_problem",
           "legendre_project_cell", "legendre_project_face"]
