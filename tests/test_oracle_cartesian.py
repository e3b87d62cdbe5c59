"""Pins of the oracle's Cartesian-summation route (Eq. 3-6, CPU).

Brute force: the constant image's Z_00 is the count of pixel centres in the
disk times the pixel area over pi (counted with integers), and a 4 x 4 image
summed by hand.  Invariants: the pixel-centre set of a square image with a
centred disk is symmetric under quarter turns and mirrors, so rot90 multiplies
Z_nm by (-i)^m and a vertical flip conjugates it, and the constant image has
Z_nm = 0 unless 4 divides m.  Consistency: for a smooth image the Cartesian
and polar quadratures of Eq. 1 agree to their discretisation error.
"""

import numpy as np
import pytest

from oracle import cartesian, grid, moments, zernike
from paper_2304_14492_gb300 import synth


@pytest.mark.parametrize("n", [4, 63, 64, 101])
def test_constant_image_z00_counts_disk_pixels(n):
    # x = (2c + 1 - N)/N: inside iff (2c + 1 - N)^2 + (2r + 1 - N)^2 <= N^2
    count = sum(1 for r in range(n) for c in range(n) if (2 * c + 1 - n) ** 2 + (2 * r + 1 - n) ** 2 <= n * n)
    pairs = [(0, 0)] + [(k, k % 2) for k in range(1, 9)] + [(6, 2), (8, 4), (9, 5), (12, 8), (7, 7)]
    z = cartesian.moments_cartesian(np.ones((n, n)), pairs)
    assert abs(z[0] - count * 4.0 / (np.pi * n * n)) <= 1e-13
    for (nn, m), v in zip(pairs, z):
        if m % 4:
            assert abs(v) <= 1e-12, (nn, m)


def test_four_by_four_by_hand():
    # centre (1.5, 1.5), r = 2: offsets +-0.5, +-1.5; the four corners
    # (|u| = |v| = 1.5) fall outside; Z_11 = 2/pi * (1/4) * sum f (x - j y)
    img = np.arange(16, dtype=np.float64).reshape(4, 4) + 1.0
    want11 = 0.0
    want20 = 0.0
    for row in range(4):
        for col in range(4):
            u, v = col - 1.5, 1.5 - row
            if u * u + v * v <= 4.0:
                x, y = u / 2.0, v / 2.0
                want11 += img[row, col] * (x - 1j * y)
                want20 += img[row, col] * (2.0 * (x * x + y * y) - 1.0)
    z = cartesian.moments_cartesian(img, [(1, 1), (2, 0)])
    assert abs(z[0] - 2.0 / np.pi * 0.25 * want11) <= 1e-13
    assert abs(z[1] - 3.0 / np.pi * 0.25 * want20) <= 1e-13


@pytest.mark.parametrize("n", [32, 33])
def test_quarter_turn_and_mirror(n):
    img = synth.uniform_image(n, n, workload=21, index=n)
    pairs = [(nn, m) for nn in range(0, 13) for m in range(nn % 2, nn + 1, 2)]
    z = cartesian.moments_cartesian(img, pairs)
    zr = cartesian.moments_cartesian(np.rot90(img), pairs)          # counter-clockwise
    zf = cartesian.moments_cartesian(np.flipud(img), pairs)         # y -> -y
    for k, (nn, m) in enumerate(pairs):
        assert abs(zr[k] - (-1j) ** m * z[k]) <= 1e-12 * max(1.0, abs(z[k]))
        assert abs(zf[k] - np.conj(z[k])) <= 1e-12 * max(1.0, abs(z[k]))


def test_agrees_with_the_polar_quadrature_on_a_smooth_image():
    n = 256
    yy, xx = np.mgrid[0:n, 0:n]
    img = np.exp(-((xx - 140.0) ** 2 + (yy - 110.0) ** 2) / (2 * 30.0 ** 2))
    pairs = [(0, 0), (2, 0), (3, 1), (4, 2), (6, 4), (10, 6)]
    zc = cartesian.moments_cartesian(img, pairs)
    zp_all = moments.moments(img, 10, 128, 256, grid="gauss")
    zp = np.array([zp_all[zernike.moment_index(nn, m)] for nn, m in pairs])
    assert np.max(np.abs(zc - zp)) <= 3e-4 * np.max(np.abs(zp))


def test_disk_pixels_geometry():
    rows, cols, x, y = cartesian.disk_pixels(4, 4)
    assert len(rows) == 12
    assert np.all(x * x + y * y <= 1.0)
    cx, cy, r = grid.default_geometry(4, 4)
    assert (cx, cy, r) == (1.5, 1.5, 2.0)
