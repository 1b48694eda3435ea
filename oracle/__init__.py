"""Plain, slow, FP64 CPU oracle for BST filtered backprojection.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA
kernels (no kernels, headers, tables or helpers); the two meet only through
the seeded input generators of ``synth``.

Modules
-------
brute    Eq. 2 backprojection B as a Riemann sum with linear interpolation
         (the slant-stack "SS" of Sec. 2), its transpose R (Eq. 1 discretised
         as the exact adjoint), and SS filtered backprojection.
bst      The BST method of Sec. 2 (Theorem 2.1, Eq. 3) step by step in the
         paper's stage order P0..P8: centre-aligned zero padding, 1D FFT
         along rays, the filter / 1/sigma weight, polar-to-Cartesian bilinear
         gridding in the Fourier domain, 2D inverse FFT, crop (fftshift) and
         scale.  A direct-DFT mode replaces the FFTs by explicit sums.
kb       Stage P5 as Kaiser-Bessel convolution gridding (polar samples weighted
         by their cell area, spread with a separable KB kernel, inverse FFT,
         division by the kernel's transform), and the direct sum over polar
         samples that it approximates.
prep     The pre-reconstruction stages: normalization, centering, window P1.
adjoint  The exact adjoint of the discrete BST operator (a Fourier-slice
         projector, the "FST" dual of Sec. 2) and the gradient of
         ||FBP(p; g) - f||^2 with respect to the filter taps g.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(closed forms, invariants, brute force on tiny inputs, adjoint identities and
finite differences).  The paper prints no worked numerical example, so no
value is pinned to a number printed in the paper.
"""
