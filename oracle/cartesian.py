"""Zernike moments by Cartesian summation (oracle; test infrastructure only).

Sec. 2, Eq. 3-6: instead of interpolating the image onto a polar grid, the
moment integral is approximated by a sum over the pixels whose centres lie in
the unit disk, each pixel weighted by its area Delta^2 (the first-order
approximation of Eq. 5):

    Z_nm = (n + 1)/pi * sum_{pixels in the disk} Delta^2 R_nm(rho) f(x, y) e^{-j m theta}

with (x, y) the pixel centre in disk units, rho = |(x, y)|, theta the angle of
(x, y) (Eq. 6 prints "y/x": read as atan2 with the y axis up, the same reading
as the polar route).  Reading of the prefactor: Eq. 6 prints 1/(pi N^2) while
Eq. 5 gives Delta = 2/N for an N x N image, i.e. Delta^2 = 4/N^2; this oracle
keeps Eq. 3-5 (Delta^2 = 1/r^2 for a disk of radius r pixels, 4/N^2 when the
disk is inscribed in an N x N image).

Geometry as on the polar route: pixel centres on integer coordinates, disk
centre (cx, cy) and radius r in pixels, x = (col - cx)/r, y = (cy - row)/r.
The radial polynomials come from the Jacobi recurrence (``zernike.zrp``); the
sum is taken directly over every pixel (no symmetry folding).
"""

import numpy as np

from .grid import default_geometry
from .zernike import zrp


def disk_pixels(height, width, geometry=None):
    """(rows, cols, x, y) of the pixel centres with x^2 + y^2 <= 1."""
    cx, cy, r = geometry if geometry is not None else default_geometry(height, width)
    rows, cols = np.mgrid[0:height, 0:width]
    x = (cols - cx) / r
    y = (cy - rows) / r
    inside = x * x + y * y <= 1.0
    return rows[inside], cols[inside], x[inside], y[inside]


def moments_cartesian(img, pairs, geometry=None):
    """Z_nm of Eq. 6 (prefactor per Eq. 3-5) for each (n, m) in ``pairs``;
    complex128 array in the order of ``pairs``."""
    img = np.asarray(img, dtype=np.float64)
    h, w = img.shape
    geo = geometry if geometry is not None else default_geometry(h, w)
    rows, cols, x, y = disk_pixels(h, w, geo)
    f = img[rows, cols]
    rho = np.sqrt(x * x + y * y)
    theta = np.arctan2(y, x)
    area = 1.0 / (geo[2] * geo[2])                      # Delta^2 in disk units
    out = np.empty(len(pairs), dtype=np.complex128)
    for k, (n, m) in enumerate(pairs):
        ker = zrp(n, m, rho) * np.exp(-1j * m * theta)
        out[k] = (n + 1) / np.pi * area * np.sum(f * ker)
    return out
