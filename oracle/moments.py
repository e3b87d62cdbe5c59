"""Zernike moments on the polar grid (oracle; test infrastructure only).

Eq. 1: Z_nm = (n+1)/pi * integral of f_hat(rho, theta) R_nm(rho) e^{-j m theta}
rho d rho d theta over the unit disk.  Discretised on the polar grid:

    F_m(rho_i) = sum_k f_hat(rho_i, theta_k) e^{-j m theta_k}          (angular)
    Z_nm       = (n+1)/pi * sum_i wr_i (2 pi / N_theta) R_nm(rho_i) F_m(rho_i)

The angular sum is done as a plain DFT (no FFT), the radial polynomials come
from ``zernike.zrp_table`` (no Eq. 7).  Eq. 14-15: with the Neumann option the
moment is divided by eps_m = 2 for m = 0 and 1 otherwise.
"""

import numpy as np

from .grid import default_geometry, radial_nodes
from .resample import polar_resample
from .zernike import index_pairs, zrp_table


def neumann_factor(m):
    """eps_m of Eq. 15."""
    return 2.0 if m == 0 else 1.0


def angular_dft(fhat, n_max):
    """F[i, m] = sum_k fhat[i, k] e^{-2 pi j m k / N_theta}, m = 0..n_max.

    The exponent's angle is reduced exactly as (m k mod N_theta) before the
    cosine and sine are taken, so the DFT matrix is exactly periodic."""
    fhat = np.asarray(fhat, dtype=np.float64)
    n_theta = fhat.shape[-1]
    k = np.arange(n_theta)[:, None]
    m = np.arange(n_max + 1)[None, :]
    ang = 2.0 * np.pi * ((m * k) % n_theta) / n_theta
    dft = np.cos(ang) - 1j * np.sin(ang)
    return fhat @ dft


def project(F, wr, n_theta, n_max, table=None, rho=None, neumann=False):
    """Radial quadrature of Eq. 1 for every stored (n, m): returns complex Z of
    length P(n_max) in ``index_pairs`` order.  ``F`` is [N_rho, >= n_max+1]."""
    if table is None:
        table = zrp_table(n_max, rho)
    pairs = index_pairs(n_max)
    Z = np.zeros(len(pairs), dtype=np.complex128)
    dtheta = 2.0 * np.pi / n_theta
    for row, (n, m) in enumerate(pairs):
        z = (n + 1) / np.pi * np.sum(wr * dtheta * table[row] * F[:, m])
        if neumann:
            z = z / neumann_factor(m)
        Z[row] = z
    return Z


def moments_polar(fhat, n_max, grid="midpoint", neumann=False):
    """Moments of a function already sampled on the polar grid:
    fhat[N_rho, N_theta] on ``radial_nodes(N_rho, grid)`` x ``angles``."""
    fhat = np.asarray(fhat, dtype=np.float64)
    n_rho, n_theta = fhat.shape
    rho, wr = radial_nodes(n_rho, grid)
    F = angular_dft(fhat, n_max)
    return project(F, wr, n_theta, n_max, rho=rho, neumann=neumann)


def moments(img, n_max, n_rho, n_theta, grid="midpoint", neumann=False, geometry=None):
    """Zernike moments of a Cartesian image: bilinear polar resampling, then
    ``moments_polar``.  Default geometry: the disk inscribed in the image."""
    img = np.asarray(img, dtype=np.float64)
    if geometry is None:
        geometry = default_geometry(*img.shape)
    rho, _ = radial_nodes(n_rho, grid)
    fhat = polar_resample(img, rho, n_theta, geometry)
    return moments_polar(fhat, n_max, grid, neumann)
