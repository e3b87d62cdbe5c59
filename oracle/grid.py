"""Polar grid and image geometry (oracle; test infrastructure only).

Sec. 2.5: the polar integral of Eq. 1 is evaluated by sampling rho in (0, 1)
and theta in [0, 2 pi) uniformly and interpolating the image there.  The paper
does not fix the radial rule; this oracle takes the midpoint rule
rho_i = (i + 1/2)/N_rho with weight rho_i / N_rho (the Jacobian rho of Eq. 1
folded in), and offers Gauss-Legendre nodes on [0, 1] as the exact rule.
"""

import numpy as np


def radial_nodes(n_rho, kind="midpoint"):
    """Radial nodes rho_i and weights wr_i with sum_i wr_i g(rho_i) ~ the
    integral of g(rho) rho d rho over [0, 1]."""
    if n_rho < 1:
        raise ValueError("n_rho >= 1")
    if kind == "midpoint":
        rho = (np.arange(n_rho, dtype=np.float64) + 0.5) / n_rho
        wr = rho / n_rho
    elif kind == "gauss":
        x, w = np.polynomial.legendre.leggauss(n_rho)
        rho = (x + 1.0) / 2.0
        wr = w / 2.0 * rho
    else:
        raise ValueError(kind)
    return rho, wr


def angles(n_theta):
    """theta_k = 2 pi k / N_theta, k = 0..N_theta-1."""
    return 2.0 * np.pi * np.arange(n_theta, dtype=np.float64) / n_theta


def default_geometry(height, width):
    """Unit disk inscribed in the image: centre at the middle of the pixel
    grid (pixel centres sit on integer coordinates), radius min(H, W)/2 px."""
    return (width - 1) / 2.0, (height - 1) / 2.0, min(height, width) / 2.0


def polar_to_pixel(rho, theta, geometry):
    """Pixel coordinates (X, Y) of the polar point (rho, theta); theta runs
    counter-clockwise with the y axis pointing up, so rows grow downwards."""
    cx, cy, r = geometry
    return cx + r * rho * np.cos(theta), cy - r * rho * np.sin(theta)


def pixel_to_polar(x, y, geometry):
    """(rho_xy, theta_xy) of pixel centres, theta in [0, 2 pi) (Eq. 9 uses
    theta_xy; the extracted text's "y/x" is read as atan2 with y up)."""
    cx, cy, r = geometry
    dx = np.asarray(x, dtype=np.float64) - cx
    dy = cy - np.asarray(y, dtype=np.float64)
    rho = np.sqrt(dx * dx + dy * dy) / r
    theta = np.mod(np.arctan2(dy, dx), 2.0 * np.pi)
    return rho, theta
