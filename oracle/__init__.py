"""CPU oracle for the MGRIT / semi-Lagrangian method (De Sterck, Falgout, Krzysik 2022).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 numpy
restatement of the paper's method, written to check the CUDA path.  Only the
test suite, the smoke check and the benchmark's CPU-baseline leg may import it;
the library never does, and the library has no CPU fallback.

It shares no code with the CUDA path: no kernels, headers, helper functions or
constant tables.  Inputs come from the separate `workloads` module.

Modules (each function cites the passage of the paper it follows):
  semi_lagrangian  grid, wave speeds, ERK departure points, east-neighbour
                   decomposition, Lagrange weights, the SL step (Sec. 2.1, Sec. 4.1)
  coarse           D_{p+1}, f_{p+1}, backtracking, phi / sigma, the corrected
                   coarse operator Psi (Sec. 3, Sec. 4.2, Sec. SM6)
  mgrit            sequential time stepping and the linear FCF MGRIT V-cycle (Sec. 2.2)
  fourier          Fourier symbols and the two-level estimate rho(c) (Sec. 2.3)
  adjoint          explicit transposed operators and the discrete adjoint

Parity status: every function is pinned by a `-m "not gpu"` test except those
whose header says "parity unpinned".
"""
