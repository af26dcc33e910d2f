"""CPU FP64 oracle for the matrix-free Q4 stream-function solve (TEST INFRASTRUCTURE ONLY).

This package is the independent, slow, obviously-correct statement of what the
GPU library computes.  It is used by `tests/`, by `__graft_entry__.smoke()` and by
the CPU-baseline leg of `bench.py`, and by nothing else: the library itself never
imports it, and it imports nothing from the library.  It shares no arithmetic with
the CUDA path; the only shared module is the seeded geometry generator
`paper_2512_12232_gb300.workloads`, which the tests call to produce inputs for both.

Everything is float64 (numpy / scipy).  Each function cites the passage of
Sadasivan & Yadav, "A Computational Approach for Multi-Body Potential-Flow
Interaction Effects Using Matrix-Free FEM and Body-Conforming Grids" that it
follows:

* `mesh`    - body-conforming grid generation (section "Body-Conforming Grid
              Generation": displacement of near-boundary nodes, Laplacian
              propagation of the displacement, x_new = x_old + d).
* `element` - Q4 element stiffness K_e = int (grad N)^T grad N (section
              "Weak formulation").
* `system`  - unknown set N_dof = N_int + N_N + N_b and the reduced system with one
              multi-point-constraint unknown per body (section "Matrix-Free Conjugate
              Gradient with Multiple Constraint Enforcement").
* `solve`   - direct solve (the definition of the discrete solution), the CG of
              Appendix A (Algorithm, element-by-element), and the body Schur form.
* `post`    - surface tangential velocity (section "Velocity Field and Surface
              Tangential Velocity") and Q / CoPFI (section "Effect of Gap Ratio").
* `cutmesh` - the mixed-cell variant of the grid generation: surface points where grid
              edges cross the body boundary (circles and polygons), node splitting,
              triangle / pentagon cells
              (pentagon = triangle + quadrilateral), boundary-point redistribution,
              and the cut-cell element matrices and outputs.
* `grad`    - adjoint shape gradient of CoPFI / gap flow (beyond the paper; its
              conclusions name sensitivity analysis and shape optimisation).

Pins (tests/test_oracle_*.py, all `-m "not gpu"`): textbook closed-form rectangle
stiffness, element invariants (zero row sums, symmetry, PSD with constant
nullspace, rigid-motion and scale invariance), brute-force loop versions of the
mesh rules on tiny grids, the linear patch test, the closed-form cylinder
psi = U y (1 - a^2/r^2) with second-order convergence, symmetry invariants of the
paper's Table 1 layout, flux balance, dense-vs-sparse-vs-CG agreement, Schur vs
MPC, central finite differences of the gradient, and for the mixed-cell mesh hand-built
split layouts, the right-triangle stiffness, the tiling-area identity, the piece-wise
patch test and closed-form cylinder convergence.  The paper's Table 1 numbers
themselves are "parity unpinned": its cylinder x-positions are only in figures.
"""
