"""Reconstruction errors and normalisation (oracle; test infrastructure only).

Sec. 2.4: Eq. 10 (relative squared error) and Eq. 13 (squared error over the
squared maximum grey level times the number of pixels), both over the pixels
with x^2 + y^2 <= 1.  Sec. 3 / Table I: the reconstruction is mapped linearly
onto [min f, max f] of the original.  Readings: the pixel count of Eq. 13's
denominator is the number of pixels inside the disk; f_max, min and max are
taken over the disk pixels.
"""

import numpy as np

from .grid import default_geometry, pixel_to_polar


def disk_mask(height, width, geometry=None):
    """Pixels whose centre lies in the closed unit disk."""
    if geometry is None:
        geometry = default_geometry(height, width)
    y, x = np.mgrid[0:height, 0:width]
    rho, _ = pixel_to_polar(x, y, geometry)
    return rho <= 1.0


def eps1(f, ftilde, mask):
    """Eq. 10: sum (f - f~)^2 / sum f^2 over the mask."""
    f = np.asarray(f, dtype=np.float64)[mask]
    g = np.asarray(ftilde, dtype=np.float64)[mask]
    return float(np.sum((f - g) ** 2) / np.sum(f ** 2))


def eps13(f, ftilde, mask):
    """Eq. 13: sum (f - f~)^2 / (f_max^2 * number of pixels) over the mask."""
    f = np.asarray(f, dtype=np.float64)[mask]
    g = np.asarray(ftilde, dtype=np.float64)[mask]
    return float(np.sum((f - g) ** 2) / (np.max(f) ** 2 * f.size))


def minmax_normalize(ftilde, lo, hi, mask):
    """Map f~ linearly so that its min / max over the mask become lo / hi
    (Table I); pixels outside the mask stay zero."""
    g = np.asarray(ftilde, dtype=np.float64)
    gmin = g[mask].min()
    gmax = g[mask].max()
    scale = (hi - lo) / (gmax - gmin) if gmax > gmin else 0.0
    out = lo + (g - gmin) * scale
    return np.where(mask, out, 0.0)


def rel_max_err(Z, Zref):
    """max |Z - Zref| / max |Zref|: the parity measure of a moment vector."""
    Z = np.asarray(Z)
    Zref = np.asarray(Zref)
    return float(np.max(np.abs(Z - Zref)) / np.max(np.abs(Zref)))
