"""FP64 CPU oracle for randomized block orthogonalization and s-step GMRES.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` may use it.  It is a plain, slow, step-by-step restatement
of the schemes of Yamazaki, Higgins, Boman and Szyld, "Random sketching to
enhance the numerical stability of block orthogonalization algorithms for
s-step GMRES" (arXiv 2503.16717), in float64.  It shares no code with the
CUDA library.

Two implementations of the same definitions: the numpy modules below, and a plain
C++17 implementation in ``cpp/`` (loops over column-major float64 arrays, no BLAS;
built by ``build_cpp.py``, bound by ``cpp_oracle.py``) of the sketch, the dense
kernels, the accuracy measures, the one-stage and two-stage schemes, CSR SpMV,
s-step GMRES with the monomial basis and Householder GMRES.  The GPU parity tests of
the orthogonalization schemes and ``smoke()`` check against the C++ one; the numpy
one covers what the C++ one does not (Newton and Chebyshev bases, Gaussian and
Count-Gauss sketch schemes, the learned preconditioner), and the two are checked
against each other in ``tests/test_oracle_cpp.py``.

Modules
-------
sketch   sparse-sign sketch from the SplitMix64 stream (Section 3; "sparse
         dimension reduction maps"), hash indices/signs and the sketch apply;
         Gaussian and Count-Gauss sketches (Section 5.2).
dense    small dense kernels: upper Cholesky with breakdown detection,
         Householder QR with non-negative diagonal, triangular solves.
orth     BCGS, CholQR, CholQR2, RandHH, RandCholQR, one-stage BCGS2
         (Figures 2-4, Section 5) and the two-stage scheme with RandBCGS2 or
         BCGS-PIP preprocessing (Figures 5-7, Section 7, Appendix).
metrics  ||I - Q^T Q||_2 and ||V - QR||_2 / ||V||_2 evaluated in extended
         precision (equations (1), (2)-(3)).
krylov   CSR SpMV, monomial, Newton (Leja-ordered Ritz values) and Chebyshev
         (smallest-capacity ellipse) matrix-powers bases, s-step GMRES
         (Figure 1, Section 4) and Householder-Arnoldi GMRES (Walker 1988) as
         the brute-force reference.
gnn      the learned sparse-approximate-inverse preconditioner of the workload
         (not in the paper): graph network, loss, gradient, Adam, and the
         classical SPAI minimiser as its pin.

Parity status: every function has a pin in ``tests/test_oracle_*.py``
(closed forms, library special cases, paper-stated invariants).  The
absolute GMRES iteration counts of the PDE workloads are "parity unpinned":
the paper prints counts only for a 300^3 problem with an unstated right-hand
side and preconditioner.
"""
