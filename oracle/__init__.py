"""FP64 CPU oracle of Coprime Blurred Pair (CBP) deblurring -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it and shares no code with it.

Method: Thorpe, Li, Li, Yu, Saunders, Yu, "A Co-Prime Blur Scheme for Data
Security in Video Surveillance" (arXiv 1203.4874).  Each function cites the
passage it follows.  Every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, brute force, exact
arithmetic, library routines); see ``tests/test_oracle_pins.py``.  The two
diagnostics ``sigma_gap`` and ``kappa`` are reported quantities whose values
are pinned only through the singular values of a library SVD.
"""
from .cbp_oracle import (  # noqa: F401
    root_powers, blur_full, blur_pair, evaluate_z2, evaluate_z1,
    convolution_matrix, sylvester_system, null_vector, cofactors_pass,
    lift, scale_least_squares, kernel_spectra, kernels_from_spectra,
    fft_grid_size, deconvolve_dual, estimate_kernels, deblur_pair,
    plane_sums, size_ratios, estimate_size, truncate_lsb, scale_least_squares_k1,
    scale_support, kernel_spectra_support,
)
from .coprime import resultant_nonzero  # noqa: F401
from . import camera  # noqa: F401
