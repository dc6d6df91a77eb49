"""FP64 CPU oracle for the frozen Gaussian reconstruction hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's formulas (Chai & Deng, "Frozen Gaussian Grid-point
Correction For Semi-classical Schroedinger Equation").  Only the tests, the
smoke check of the package entry point and the CPU-baseline / reference leg of
the benchmark may import, call, link or execute anything in here.  The CUDA
library never calls it, and it shares no code with the library: the only
common module is the seeded input generator in ``workloads``.

Modules
-------
fga           eq. 2.10 / 2.15 / 2.16: packets, inner product, windowed direct sum
lsa           Sec. 2.2-3.2: neighbour map, eps-free Gram and right-hand side,
              SVD pseudo-inverse, Algorithms 1 and 2 coefficients, E_LSA, M_LSA
fggc          eq. 2.24-2.25: aggregation onto grid nodes and on-grid sum;
              Algorithm 3 (multi-step FGGC with a fixed mesh and learned flow)
decompose     eq. 2.6 / 2.8: initial decomposition of a wave given on the grid
trajectories  eq. 2.3-2.7: classical RK4 of Q, P, S, A with the Jacobians
              (plain C in c/rk4.c, compiled on first use)
exact         the exact Gaussian solution for V = |x|^2/2 (reference of the
              multi-step examples of Sec. 4.4)

Parity status: every function is pinned by a test in tests/test_oracle_*.py
against a closed form, a brute-force evaluation, an independent quadrature or a
value printed in the paper.
"""
