"""Pins of the oracle's reconstruction and metrics (CPU).

Eq. 9 identity for the Neumann reading (half spectrum with c_m = 2/eps_m is the
literal sum over m = -n..n), exact round trip of band-limited polar functions
on Gauss-Legendre nodes, the interpolation onto pixels on functions it must
reproduce, Eq. 10 / Eq. 13 on hand-made arrays, and the min-max normalisation
against the values printed in Table I.
"""

import os

import numpy as np

from oracle import grid, metrics, moments, reconstruct, zernike

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_moments(n_max, seed):
    rng = np.random.default_rng(seed)
    pairs = zernike.index_pairs(n_max)
    Z = rng.standard_normal(len(pairs)) + 1j * rng.standard_normal(len(pairs))
    for r, (n, m) in enumerate(pairs):
        if m == 0:
            Z[r] = Z[r].real          # Z_{n,0} is real for a real image
    return Z


def test_neumann_reading_identity():
    n_max, n_rho, n_theta = 12, 9, 32
    Z = random_moments(n_max, 3)
    rho, _ = grid.radial_nodes(n_rho)
    th = grid.angles(n_theta)
    full = reconstruct.eq9_full(Z, n_max, rho[:, None] + 0 * th[None, :], th[None, :] + 0 * rho[:, None])
    with_n = reconstruct.reconstruct_polar(Z, n_max, n_rho, n_theta, neumann=True)
    without = reconstruct.reconstruct_polar(Z, n_max, n_rho, n_theta, neumann=False)
    assert np.max(np.abs(with_n - full)) <= 1e-12
    # the half sum = (literal Eq. 9 + its m = 0 part) / 2
    table = zernike.zrp_table(n_max, rho)
    m0 = sum(Z[r].real * table[r] for r, (n, m) in enumerate(zernike.index_pairs(n_max)) if m == 0)
    assert np.max(np.abs(without - 0.5 * (full + m0[:, None]))) <= 1e-12


def test_round_trip_band_limited_gauss():
    # f = literal Eq. 9 of random moments, sampled on a Gauss-Legendre polar
    # grid with N_theta > 2 n_max: its moments are the random moments, and the
    # reconstruction returns f exactly.
    n_max, n_theta = 16, 64
    n_rho = n_max + 1
    Z = random_moments(n_max, 11)
    rho, _ = grid.radial_nodes(n_rho, "gauss")
    th = grid.angles(n_theta)
    f = reconstruct.eq9_full(Z, n_max, rho[:, None] + 0 * th[None, :], th[None, :] + 0 * rho[:, None])
    Zr = moments.moments_polar(f, n_max, "gauss")
    assert np.max(np.abs(Zr - Z)) <= 1e-12
    fr = reconstruct.reconstruct_polar(Zr, n_max, n_rho, n_theta, "gauss", neumann=True)
    assert np.max(np.abs(fr - f)) <= 1e-12


def test_polar_to_cartesian_reproduces_linear_functions():
    h = w = 40
    n_rho, n_theta = 20, 64
    rho, _ = grid.radial_nodes(n_rho)
    geo = grid.default_geometry(h, w)
    y, x = np.mgrid[0:h, 0:w]
    r_xy, t_xy = grid.pixel_to_polar(x, y, geo)
    inside = r_xy <= 1.0
    # f = rho: exact between the first and last ring, clamped outside them
    f_rho = np.repeat(rho[:, None], n_theta, axis=1)
    out = reconstruct.polar_to_cartesian(f_rho, rho, h, w)
    want = np.clip(r_xy, rho[0], rho[-1])
    assert np.max(np.abs(out[inside] - want[inside])) <= 1e-12
    assert np.all(out[~inside] == 0)
    # f = k: exact in v = theta N / 2 pi except across the wrap k = N-1 -> 0
    f_k = np.repeat(np.arange(n_theta, dtype=float)[None, :], n_rho, axis=0)
    out = reconstruct.polar_to_cartesian(f_k, rho, h, w)
    v = t_xy * n_theta / (2 * np.pi)
    sel = inside & (v < n_theta - 1)
    assert np.max(np.abs(out[sel] - v[sel])) <= 1e-9


def test_reconstruct_pixels_vs_literal_eq9():
    n_max = 8
    Z = random_moments(n_max, 5)
    h, w = 17, 23
    geo = grid.default_geometry(h, w)
    y, x = np.mgrid[0:h, 0:w]
    r_xy, t_xy = grid.pixel_to_polar(x, y, geo)
    inside = r_xy <= 1.0
    out = reconstruct.reconstruct_pixels(Z, n_max, h, w, neumann=True)
    full = reconstruct.eq9_full(Z, n_max, r_xy[inside], t_xy[inside])
    assert np.max(np.abs(out[inside] - full)) <= 1e-12
    assert np.all(out[~inside] == 0)


def test_eq10_eq13_hand_values():
    f = np.array([[1.0, 2.0], [3.0, 4.0]])
    g = np.array([[1.0, 1.0], [3.0, 6.0]])
    mask = np.array([[True, True], [False, True]])
    # squared errors over mask: 0, 1, 4 -> 5; sum f^2 over mask: 1 + 4 + 16 = 21
    assert abs(metrics.eps1(f, g, mask) - 5.0 / 21.0) <= 1e-15
    # f_max over mask = 4, count = 3
    assert abs(metrics.eps13(f, g, mask) - 5.0 / (16.0 * 3)) <= 1e-15
    assert metrics.eps1(f, f, mask) == 0.0
    assert metrics.eps1(f, 0 * f, mask) == 1.0
    assert metrics.disk_mask(64, 64).sum() == np.sum(
        (np.mgrid[0:64, 0:64][1] - 31.5) ** 2 + (np.mgrid[0:64, 0:64][0] - 31.5) ** 2 <= 32.0 ** 2)


def read_table1():
    bands = {}
    cur = None
    with open(os.path.join(GOLDEN, "table1_minmax.txt")) as fh:
        for line in fh:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "band":
                cur = bands.setdefault(t[1], {"raw": [], "norm": []})
            else:
                cur[t[0]].append([float(v) for v in t[1:]])
    return {b: (np.array(d["raw"]), np.array(d["norm"])) for b, d in bands.items()}


def test_minmax_normalisation_against_table1():
    # Table I: the normalised patch is an affine map of the raw patch per band.
    # Fit the map on the usable (non-clipped) entries, then ask the oracle to
    # map the raw patch onto the fitted images of its own min / max: it must
    # reproduce the printed values within the printing's rounding.
    for band, (raw, norm) in read_table1().items():
        use = raw > 0
        A = np.stack([np.ones(use.sum()), raw[use]], 1)
        (a, b), *_ = np.linalg.lstsq(A, norm[use], rcond=None)
        assert b > 0
        lo, hi = a + b * raw[use].min(), a + b * raw[use].max()
        mapped = metrics.minmax_normalize(np.where(use, raw, raw[use].min()), lo, hi, use)
        assert np.max(np.abs(mapped[use] - norm[use])) <= 0.75, band
    # and the normalised result spans exactly [lo, hi]
    g = np.array([[3.0, -1.0], [5.0, 2.0]])
    out = metrics.minmax_normalize(g, 10.0, 20.0, np.ones_like(g, bool))
    assert out.min() == 10.0 and out.max() == 20.0
