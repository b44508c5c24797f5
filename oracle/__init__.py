"""Plain CPU FP64 oracle for the Fourier-basis Helmholtz FMM apply.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code, table or constant generator with the CUDA library; it reads the
paper (Cecka & Darve, "Fourier Based Fast Multipole Method for the Helmholtz
Equation", arXiv 0911.4114) and nothing else.

Modules
-------
direct      Eq. (HelmholtzMatrixVector): the O(N*M) direct sum, its adjoint and
            the position gradient of a quadratic loss (ground truth).
tree        Section 2 (octree, interaction list, neighbour list) under the
            tree conventions stated in that module.
quadrature  Sections 2.1, 3.1-3.4: truncation l (Eq. EBF + Eq. CollinoError),
            N_theta (Algorithm Ntheta), N_phi(theta_n) (Algorithm Nphi), the
            band-limited modified transfer function (Algorithm BMTF), Fourier
            re-sampling and the five-step re-quadrature (Section 3.4).
fmm         Section 2 (S2M, M2M, M2L, L2L, L2T + near field, Eq. FMM_FinalStep)
            on the Fourier quadratures of Section 3, step by step.

Every function runs in float64 / complex128.  Library primitives used as
single steps: numpy FFT, numpy matmul, scipy spherical Bessel / Bessel /
Legendre functions.  Functions whose result has no independent pin say
"parity unpinned" in their docstring (none at present).
"""
