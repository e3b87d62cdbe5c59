"""Bilinear polar resampling f -> f_hat(rho, theta) (oracle; test infrastructure
only).

Sec. 2.5: the polar form f_hat of Eq. 1 is obtained by interpolating the
Cartesian image at uniformly spaced (rho, theta).  The interpolation kind is
bilinear; samples whose neighbours fall outside the image take zero there,
which is the zero embedding the paper uses (Sec. 3, the image placed inside a
zero-valued grid).
"""

import numpy as np

from .grid import angles, default_geometry, polar_to_pixel


def pixel(img, x, y):
    """img[y, x] for integer arrays x, y, and 0 outside the image."""
    h, w = img.shape
    inside = (x >= 0) & (x < w) & (y >= 0) & (y < h)
    out = np.zeros(np.broadcast(x, y).shape, dtype=np.float64)
    out[inside] = img[y[inside], x[inside]]
    return out


def bilinear(img, X, Y):
    """Bilinear interpolation at real pixel coordinates (X = column, Y = row):
    the four neighbours floor(X)..floor(X)+1 by floor(Y)..floor(Y)+1 weighted
    by the fractional offsets."""
    img = np.asarray(img, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    x0 = np.floor(X).astype(np.int64)
    y0 = np.floor(Y).astype(np.int64)
    fx = X - x0
    fy = Y - y0
    return ((1 - fx) * (1 - fy) * pixel(img, x0, y0)
            + fx * (1 - fy) * pixel(img, x0 + 1, y0)
            + (1 - fx) * fy * pixel(img, x0, y0 + 1)
            + fx * fy * pixel(img, x0 + 1, y0 + 1))


def polar_resample(img, rho, n_theta, geometry=None):
    """f_hat[i, k] = bilinear(img) at (rho_i, theta_k), shape [len(rho), N_theta]."""
    img = np.asarray(img)
    if geometry is None:
        geometry = default_geometry(*img.shape)
    theta = angles(n_theta)
    X, Y = polar_to_pixel(np.asarray(rho)[:, None], theta[None, :], geometry)
    return bilinear(img, X, Y)
