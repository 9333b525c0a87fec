"""Plain FP64 CPU oracle for the fast force-coupling method (Su & Keaveny, 2023).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links
this package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it. It shares no code with the CUDA path; the two meet
only through the seeded input generators, which hold none of the method's
arithmetic.

Modules
-------
closed_forms
    Gaussian kernel, the flow tensors S, Q, T, R, P, K (Sections 2.2, 3.2, 3.4),
    the FCM and modified pair mobilities, the pairwise corrections (correction
    VF / WF / WT equations) and the self corrections (Appendix B).
spectral_sum
    Direct periodic Fourier sum of the FCM mobility (the definition behind
    Appendix A, evaluated over the reciprocal lattice) for tiny N.
grid_fcm
    The grid algorithm of Section 2.1 (spread, FFT Stokes solve, trapezoidal
    interpolation), with either the FCM Gaussians (standard FCM) or the modified
    kernel of Section 3 plus the pairwise correction of Section 4 (fast FCM).
fft
    The unnormalised discrete Fourier transform and its inverse, written out
    as a mixed-radix Cooley-Tukey recursion (prime lengths by the definition);
    the grid Stokes solve and the Brownian grid noise use it.
params
    Window rule, cutoff-radius rule and grid-support rule used by both the
    standard and the fast oracle.
brownian
    Brownian increments by positive splitting (Section 3.3): grid noise through
    the square root of the Stokes operator, and the exact square root of the
    pairwise correction.
rigid
    Mobility problem of rigid bodies made of FCM particles (Section 6.1): the
    saddle-point system solved densely, and Broyden's method started from the
    diagonal-mobility Jacobian.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
a route that does not go through this package (Fourier quadrature, closed-form
lattice sums, moments, brute force, printed values); none is "parity unpinned".
"""
