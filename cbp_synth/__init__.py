"""Seeded synthetic inputs for the Coprime Blurred Pair (CBP) workloads.

This module is shared by the tests, the benchmark and the oracle's callers.  It
draws latent frames, blur kernels and noise; it holds none of the deblurring
method's arithmetic (no polynomial evaluation, no cofactor solve, no scale fix,
no deconvolution).  The blur itself (Eq. 1) is applied elsewhere: by the oracle
in tests, by the library's own forward-model kernel in the benchmark.

The paper's own videos (Point Grey Flea2 captures, 640x480, kernels 9..25,
Section 6) are not available; these generators stand in for them.

Generators (all from ``numpy.random.Generator(PCG64(seed))``):

* ``blob_latent``   -- sum of 20 Gaussian blobs (amplitude U[0,1], sigma
  U[2,10] px, centre uniform over the frame) plus a U[0,0.05] floor per pixel.
  Each blob is evaluated inside a window of radius ceil(8 sigma) around its
  centre (outside it the blob is below exp(-32) of its peak).
* ``uniform_kernel`` -- t x t entries U[0,1], normalised to sum 1.
* ``mixture_kernel`` -- w*G + (1-w)*Mo, w ~ U[0.3,0.7]; G an anisotropic
  centred Gaussian (sigma_x, sigma_y ~ U[t/6, t/3], angle U[0,pi)); Mo a random
  walk of 4t unit steps from the centre with heading drift N(0, 0.5 rad),
  bilinearly splatted and clipped to the box; normalised to sum 1.
* ``draw_kernel_pair`` -- redraws until the pair passes ``pair_is_coprime``,
  the generator's acceptance test: at every unit-circle sample used by both
  evaluation orders, the two univariate kernel polynomials keep full degree
  (one of the leading coefficients is non-zero) and share no root (their root
  sets are separated).  Section 3 requires coprime kernels.
"""
from .generators import (  # noqa: F401
    blob_latent, uniform_kernel, mixture_kernel, draw_kernel_pair,
    pair_is_coprime, gaussian_noise,
)
from .configs import (  # noqa: F401
    CONFIGS, PairInputs, make_pair_inputs,
)
