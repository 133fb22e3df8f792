"""CPU FP64 oracle for the lattice Basic Scheme (Bergmann & Merkert, arXiv 1605.05712).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's method in numpy float64.  It exists to check the
CUDA implementation in ``paper_1605_05712_gb300``; the two share no code.
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path
never calls it and has no CPU fallback.

Modules
-------
lattice     Smith normal form, pattern P(M), generating set G(M^T)  (Sec. 2.1-2.2)
transform   Fourier matrix F(M): naive definition and separable FFT (Eq. Fouriermatrix)
elasticity  isotropic stiffness, double contraction, Green operator  (Sec. 3.1)
scheme      Algorithm 1, the fixed-point scheme on patterns          (Sec. 3.2),
            and the accelerated schemes of Sec. 6 (Eyre-Milton, conjugate gradients)
analytic    laminate and generalized Hashin closed forms            (Sec. 4)
classic     independent Moulinec-Suquet scheme on a tensor grid     (Sec. 3.2, M diagonal)

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against a closed form, an invariant, brute force or a printed value of the
paper; none is "parity unpinned".
"""
