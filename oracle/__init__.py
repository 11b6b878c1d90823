"""FP64 CPU oracle for the block omega-circulant preconditioned all-at-once solver
(Fung & Hon, "Block omega-circulant preconditioners for parabolic optimal control problems").

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
(and --impl reference) leg may import this package.  It shares no code with the CUDA path and
imports nothing from it; both sides draw their inputs from the separate `synth` module.

Everything here is plain NumPy/SciPy in float64, written to be checked against the paper by eye:
library primitives (FFT, DST, sparse/dense solves, eigendecompositions) serve as single steps,
with no blocking, fusion or reordering beyond what the paper's definitions state.

Parity status per function (what pins it, see tests/test_oracle_pins.py):
  discretisation.*      pinned: sparse direct solve of the paper's block system (Sec. 1) and the
                        Example-1 errors e_h and iteration counts of Table 1 (Crank-Nicolson).
                        For theta != 1/2 the time level paired with each g and f sample in the
                        right-hand side follows the printed g~, f~ formulas and is pinned only by
                        consistency (first-order convergence): partially pinned.
  operators.matvec_*    pinned: dense A built from Eq. (matrix_A) / (matrix_A_hat), |A|^{-1}A = +-1
                        (Prop. 3.2), sparse direct solve round trip.
  spectra.*             pinned: dense omega-circulant eigendecomposition (Eq. decompositiob_S12),
                        Lemma 3.4 closed form, DST orthogonality and K S = S diag(kappa).
  precond.apply_abs_ps_inv, apply_ps_inv, apply_pms_inv
                        pinned: dense constructions of |P_S|, P_S, P_MS (Eqs. matrix_P,
                        matrix_P_GMRES, matrix_P_MS); Prop. 3.1 rank bound; Thm 3.3 clustering;
                        Thm 3.11 / Remark 4 spectral bounds.
  precond.apply_mg_ps_inv
                        pinned: Lemma 3.14 decomposition (scalar 2x2 check); with many V-cycles it
                        converges to apply_ps_inv on a = 1 (the paper's exact route).
  multigrid.*           the paper names a multigrid V-cycle but does not specify it; the reading
                        (damped Jacobi 4/5, full weighting, bilinear prolongation, averaged coarse
                        edge coefficients, nu1 = nu2 = 2) is pinned part by part
                        (tests/test_oracle_multigrid.py): Jacobi mode multipliers and the
                        smoothing factor 3/5 of local Fourier analysis, exact transfer of bilinear
                        functions, coarse coefficients of an affine a(x), the finest operator
                        against the assembled K, and the two-grid operator (and the two-level
                        V-cycle) against its 4 x 4 Fourier block analysis; the whole V-cycle also
                        converges to the exact shifted solve with a grid-independent contraction.
                        Against the paper's own multigrid numbers: Table 3 (Example 2, variable
                        a) is reproduced in iteration counts at h = 2^-5 for every gamma and for
                        MINRES-P_MS at 2^-6 and 2^-7 (tests/test_oracle_example2.py); where counts
                        differ the paper's one-sided Gauss-Seidel cycle and this symmetric
                        Jacobi cycle are different operators (the paper leaves it unspecified).
  krylov.*              pinned: sparse direct solve; Table 1 iteration counts.  The optional stall
                        exit (solves asked below float64's attainable accuracy) is checked to
                        leave reachable solves unchanged.
  finite elements (Problem(fem=True): discretisation.mass_1d, stiffness_1d, apply_M*, the M^{+-1/2}
  change of variables; spectra.mass_eigenvalues, kappa_fem)
                        pinned: element-by-element assembly of the linear and bilinear element
                        matrices, the sine eigenbasis with textbook eigenvalues, a sparse direct
                        solve of the unsymmetrised element system, dense preconditioners, and
                        Table 1's counts with elements (tests/test_oracle_fem.py).
  reference_solutions.* writes the stored FP64 solution samples (tests/golden/solution_sample_*);
                        a fresh solve of the smallest sampled instance reproduces its sample.
  Neumann route (Problem(bc="neumann"): discretisation.apply_K / K_sparse, spectra.kappa_neumann,
  spectra.dct1_*, precond.apply_ps_inv)
                        pinned: the 1D stencil written out by hand, its cosine eigenbasis,
                        dense A_hat and P_S with the nonsymmetric K as printed, a sparse direct
                        solve, and all ten rows of Table 4 (Example 3: iteration counts and e_h).
"""
from . import discretisation, operators, spectra, precond, multigrid, krylov  # noqa: F401
