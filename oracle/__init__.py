"""FP64 CPU oracle for FFT-based Zernike moments (Al-Rawi, "Ultra-Fast Zernike
Moments using FFT and GPU", arXiv 2304.14492).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link
or execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, tables, constants or helpers with the CUDA library; the two meet only
through seeded inputs that the caller passes in.

What it computes is the plain definition of the method on a polar grid, in
float64, without any FFT and without the paper's FFT identity:

* Zernike radial polynomials (ZRPs): exact rationals from the factorial sum of
  Eq. 2 (``zernike.zrp_exact``) and a stable Jacobi three-term recurrence in
  float64 (``zernike.zrp_table``).  ``zernike.zrp_eq7`` restates Eq. 7-8 (the
  paper's Chebyshev-U / DFT identity of Sec. 2.1) only so that the readings of
  that equation can be pinned against Eq. 2.
* Polar grid and bilinear resampling of the image (Sec. 2.5): ``grid``,
  ``resample``.
* Angular transform e^{-jm theta} as a direct DFT and the radial quadrature of
  Eq. 1, with the Neumann factor of Eq. 14-15: ``moments``.
* Reconstruction by Eq. 9 and the polar-to-Cartesian interpolation:
  ``reconstruct``.
* Reconstruction errors of Eq. 10 and Eq. 13 and the min-max normalisation of
  Sec. 3 / Table I: ``metrics``.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
library routines, invariants or brute force; none is marked "parity unpinned".
"""

from . import zernike, grid, resample, moments, reconstruct, metrics  # noqa: F401
