"""CPU arithmetic of the hi + lo split used by the tensor-core projection
(test helper): rounding to p significant bits, the split of a value into a
16-bit hi part and a rounded remainder, and the radial projection of Eq. 1
computed from split operands, exactly (float64 holds every product of two
16-bit values).  The weights and spectra come from the oracle."""

import numpy as np

from oracle import grid, moments as om, resample, zernike


def rne(x, p):
    """x rounded to nearest (ties to even) with p significant bits."""
    m, e = np.frexp(x)
    return np.ldexp(np.rint(np.ldexp(m, p)), e - p)


def split(x, p, lo_bits=None):
    hi = rne(x, p)
    return hi, rne(x - hi, lo_bits or p)


def terms(img, n_max, n_rho, n_theta):
    """Weights a[P, N_rho], FP32 spectra f[P, N_rho] per moment, the exact
    moments and S_nm, from the oracle."""
    rho, wr = grid.radial_nodes(n_rho)
    fh = resample.polar_resample(img.astype(np.float64), rho, n_theta, grid.default_geometry(*img.shape))
    F = om.angular_dft(fh, n_max).astype(np.complex64).astype(np.complex128)
    T = zernike.zrp_table(n_max, rho)
    pairs = zernike.index_pairs(n_max)
    a = np.array([(n + 1) / np.pi * wr * (2 * np.pi / n_theta) * T[r] for r, (n, m) in enumerate(pairs)])
    f = F[:, [m for _, m in pairs]].T
    return a, f, np.sum(a * f, axis=1), np.sum(np.abs(a) * np.abs(f), axis=1)


def split_moments(a, f, p, lo_bits=None, terms_kept=("hh", "hl", "lh")):
    ah, al = split(a, p, lo_bits)
    frh, frl = split(f.real, p, lo_bits)
    fih, fil = split(f.imag, p, lo_bits)
    fh, fl = frh + 1j * fih, frl + 1j * fil
    z = np.zeros(a.shape[0], dtype=np.complex128)
    if "hh" in terms_kept:
        z += np.sum(ah * fh, axis=1)
    if "hl" in terms_kept:
        z += np.sum(ah * fl, axis=1)
    if "lh" in terms_kept:
        z += np.sum(al * fh, axis=1)
    if "ll" in terms_kept:
        z += np.sum(al * fl, axis=1)
    return z


def dft_matrix(n_max, n_theta):
    """cos and -sin of 2 pi m k / N_theta for m = 0..n_max (the angular sums
    of Eq. 1 as a matrix product), evaluated from m k mod N_theta in float64."""
    idx = np.outer(np.arange(n_max + 1), np.arange(n_theta)) % n_theta
    ang = 2 * np.pi * idx / n_theta
    return np.cos(ang), -np.sin(ang)


def dft_split_spectra(fh, n_max, p, lo_bits=None, terms_kept=("hh", "hl", "lh")):
    """F_m(rho_i) = sum_k f_ik e^{-j m theta_k} from split samples and split
    DFT entries (f_hi w_hi + f_hi w_lo + f_lo w_hi), exactly: [N_rho, n_max + 1]."""
    c, s = dft_matrix(n_max, fh.shape[-1])
    f_hi, f_lo = split(fh, p, lo_bits)
    out = np.zeros((fh.shape[0], n_max + 1), dtype=np.complex128)
    for part, sign in ((c, 1.0), (s, 1j)):
        w_hi, w_lo = split(part, p, lo_bits)
        acc = np.zeros((fh.shape[0], n_max + 1))
        if "hh" in terms_kept:
            acc += f_hi @ w_hi.T
        if "hl" in terms_kept:
            acc += f_hi @ w_lo.T
        if "lh" in terms_kept:
            acc += f_lo @ w_hi.T
        out += sign * acc
    return out
