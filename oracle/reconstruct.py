"""Reconstruction from moments (oracle; test infrastructure only).

Eq. 9: f~(x, y) = Re sum_{n <= n_max} sum_{m = -n..n, n - m even}
Z_nm R_nm(rho_xy) e^{j m theta_xy}.  With Z_{n,-m} = conj(Z_nm) (Sec. 2) the
terms of m and -m are conjugate, so the literal sum equals
Re sum_{m >= 0} c_m Z_nm R_nm e^{j m theta} with c_0 = 1, c_{m>0} = 2.

Reading of the Neumann factor (Sec. 2.6, Eq. 14-15 and the "torchlight"
remark of Sec. 3.2): the paper's uncorrected reconstruction sums the stored
m >= 0 moments once each (c_m = 1), which over-weights the rotationally
symmetric m = 0 part; dividing by eps_m (eps_0 = 2) removes that, and the sum
becomes half of the literal Eq. 9, a scale that the min-max normalisation of
Sec. 3 removes.  Here ``neumann=True`` gives c_m = 2 / eps_m (exactly the
literal Eq. 9) and ``neumann=False`` gives c_m = 1 (the half sum).
"""

import numpy as np

from .grid import angles, default_geometry, pixel_to_polar, radial_nodes
from .moments import neumann_factor
from .zernike import index_pairs, zrp_table


def recon_weight(m, neumann):
    """c_m applied to the stored m >= 0 moment in the half-spectrum sum."""
    return 2.0 / neumann_factor(m) if neumann else 1.0


def radial_spectrum(Z, n_max, rho, neumann=False):
    """G[i, m] = sum_n c_m Z_nm R_nm(rho_i), the radial half of Eq. 9."""
    Z = np.asarray(Z, dtype=np.complex128)
    table = zrp_table(n_max, rho)
    G = np.zeros((np.size(rho), n_max + 1), dtype=np.complex128)
    for row, (n, m) in enumerate(index_pairs(n_max)):
        G[:, m] += recon_weight(m, neumann) * Z[row] * table[row]
    return G


def reconstruct_polar(Z, n_max, n_rho, n_theta, grid="midpoint", neumann=False):
    """f~ on the polar nodes, shape [N_rho, N_theta]:
    Re sum_m G[i, m] e^{j m theta_k}, with the angle m k reduced mod N_theta."""
    rho, _ = radial_nodes(n_rho, grid)
    G = radial_spectrum(Z, n_max, rho, neumann)
    k = np.arange(n_theta)[None, :]
    m = np.arange(n_max + 1)[:, None]
    ang = 2.0 * np.pi * ((m * k) % n_theta) / n_theta
    return (G @ (np.cos(ang) + 1j * np.sin(ang))).real


def eq9_full(Z, n_max, rho, theta):
    """The literal double sum of Eq. 9 over m = -n..n at points (rho, theta),
    with Z_{n,-m} = conj(Z_nm) and R_{n,-m} = R_nm."""
    Z = np.asarray(Z, dtype=np.complex128)
    rho = np.asarray(rho, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    table = zrp_table(n_max, rho.ravel())
    acc = np.zeros(rho.size, dtype=np.complex128)
    th = theta.ravel()
    for row, (n, m) in enumerate(index_pairs(n_max)):
        acc += Z[row] * table[row] * np.exp(1j * m * th)
        if m > 0:
            acc += np.conj(Z[row]) * table[row] * np.exp(-1j * m * th)
    return acc.real.reshape(rho.shape)


def polar_to_cartesian(fpolar, rho_nodes, height, width, geometry=None):
    """Bilinear interpolation of a polar image onto the pixel centres inside
    the disk (rho_xy <= 1); zero outside.

    Ring coordinate: the bracket rho_i <= rho_xy < rho_{i+1} with linear weight,
    clamped to the first / last ring below rho_0 / above rho_{N-1}.  Angle
    coordinate: v = theta_xy N_theta / (2 pi), periodic in N_theta."""
    fpolar = np.asarray(fpolar, dtype=np.float64)
    n_rho, n_theta = fpolar.shape
    if geometry is None:
        geometry = default_geometry(height, width)
    y, x = np.mgrid[0:height, 0:width]
    rho, theta = pixel_to_polar(x, y, geometry)
    nodes = np.asarray(rho_nodes, dtype=np.float64)
    i1 = np.searchsorted(nodes, rho, side="right")          # first node > rho
    i0 = np.clip(i1 - 1, 0, n_rho - 1)
    i1 = np.clip(i1, 0, n_rho - 1)
    span = nodes[i1] - nodes[i0]
    t = np.where(span > 0, (rho - nodes[i0]) / np.where(span > 0, span, 1.0), 0.0)
    t = np.clip(t, 0.0, 1.0)
    v = theta * n_theta / (2.0 * np.pi)
    k0f = np.floor(v)
    s = v - k0f
    k0 = k0f.astype(np.int64) % n_theta
    k1 = (k0 + 1) % n_theta
    val = ((1 - t) * ((1 - s) * fpolar[i0, k0] + s * fpolar[i0, k1])
           + t * ((1 - s) * fpolar[i1, k0] + s * fpolar[i1, k1]))
    return np.where(rho <= 1.0, val, 0.0)


def reconstruct_pixels(Z, n_max, height, width, geometry=None, neumann=False):
    """Eq. 9 evaluated directly at the pixel centres inside the disk (the
    half-spectrum form with c_m of ``recon_weight``); zero outside."""
    if geometry is None:
        geometry = default_geometry(height, width)
    y, x = np.mgrid[0:height, 0:width]
    rho, theta = pixel_to_polar(x, y, geometry)
    inside = rho <= 1.0
    Z = np.asarray(Z, dtype=np.complex128)
    table = zrp_table(n_max, rho[inside])
    acc = np.zeros(int(inside.sum()), dtype=np.complex128)
    th = theta[inside]
    for row, (n, m) in enumerate(index_pairs(n_max)):
        acc += recon_weight(m, neumann) * Z[row] * table[row] * np.exp(1j * m * th)
    out = np.zeros((height, width), dtype=np.float64)
    out[inside] = acc.real
    return out
