"""Plain FP64 CPU oracle for weak-constraint 4D-Var in saddle-point form.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline / reference leg may import anything from this
package.  The CUDA library shares no code with it: no kernels, headers,
helpers, constant tables or pre/post-processing.  The two meet only in the
seeded draws of ``paper_2105_06975_gb300.workload``.

Everything here is written for a reader checking it against the paper by eye
(Tabeart & Pearson, "Saddle point preconditioners for weak-constraint
4D-Var"): numpy/scipy FP64, time-major blocks, no blocking or fusion beyond
what the definitions state.  Library primitives (matmul, Cholesky, LU,
symmetric eigensolver, sparse products) serve as single steps.

Modules
-------
covariance  SOAR covariances (Sec. 6.1, Eq. SOAR) and the R-hat choices of
            Sec. 5 (diag, ridge regression Alg. 1, minimum eigenvalue Alg. 2).
model       model matrices M_i, L (Eq. def:L), L_M(k) (Definition 1), the
            L_M(k)^{-1} / ^{-T} sweeps (Lemma 1), Lorenz-96 + RK4 + tangent
            linear model (Sec. 7.1).
saddle      the saddle-point matrix A (Eq. saddlepointA), the preconditioners
            P_D and P_I (Eq. prec), their blockwise applies (Sec. 6.2), dense
            assembly, LU and the primal normal-equations check.
krylov      preconditioned MINRES, right-preconditioned GMRES and FGMRES.
problem     synthetic truth / observations / right-hand side and the
            incremental Gauss-Newton outer loop (Sec. 2.1).
bounds      Theorem 1, Remark 1, Propositions 1-4 as numbers for the pins.

Readings where the paper is silent or garbled are listed in each function's
docstring (C1..C20 in the design notes).  Parity unpinned: Table 2 values
(internally inconsistent) and the printed iteration counts (the paper's random
R_i generator and Lorenz-96 code are unavailable).
"""
