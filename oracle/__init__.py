"""Plain, slow FP64 CPU oracle for hierarchical probing of Tr(A^-1).

TEST INFRASTRUCTURE ONLY.  This package restates the method of
Stathopoulos, Laeuchli and Orginos, "Hierarchical probing for estimating the
trace of the matrix inverse on toroidal lattices" (arXiv:1302.4018), step by
step in the paper's order and notation, so that the CUDA library can be
checked against it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_1302_4018_gb300``) never imports, links or runs
anything here, and this package imports nothing from the product path; the
only code both sides share is the seeded input generator module
``paper_1302_4018_gb300.synth``, which holds no arithmetic of the method.

Modules
-------
permutation  Section 3: red-black tables (Algorithms 2, 3), the lattice
             hierarchical permutation (Algorithms 4, 5), the three-colouring
             theorem of Section 3.4 for odd factors.
probing      Section 2.2: Hadamard / Fourier matrices (Eqs. HadamardElements,
             FourierElements), the nested basis recursions
             (Eqs. Hperm-recursive, Hperm-general-recursive), the column
             sequence (Eq. HpermSequence), the direct element formula
             (Eq. row-col-permutation) and bias removal (Section 4).
operators    Section 1.1.1 / Section 5: shifted periodic Laplacian and the
             Wilson-Dirac matrix with explicit 4x4 gamma matrices and full
             3x3 link products (no spin projection, no reconstruction), the
             clover term, the even-odd Schur complement.
solvers      Textbook CG and BiCGStab in FP64 and dense solves (Section 1.1.2:
             the quadrature z^H A^-1 z is computed through a linear solve),
             Gauss and Gauss-Radau bounds from the CG coefficients.
estimator    Section 1 (Monte Carlo form of the estimator) and Section 2.2
             (nesting): quadratures q_m, prefix estimates T_s, the
             derivative of T_s with respect to a per-site mass; the
             statistics of Sections 5.2-5.3 (exact z_0-variance, speed-up
             ratio R_s, jackknife); deflation (the conclusions' next step):
             the lowest eigenpairs of the Laplacian and of gamma_5 D, the
             smallest singular triplets of D (dense decompositions), and the
             deflated quadratures written out as projected dense solves.
sparse_probing  Section 2.1, Algorithm 1 on a general sparse matrix: greedy
             colouring, Colors2Perm and the block-graph recursion, perm and
             colorOffsets, and the probing vectors of the colour paths.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against worked examples printed in the paper (``tests/golden``), closed
forms, invariants or brute force; none is marked "parity unpinned".
"""
