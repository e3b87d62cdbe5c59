"""Pins of the oracle's grid, resampler, angular transform and moments (CPU).

Closed forms: quadrature sums, the constant image (Z_00 = 1), polar Zernike
inputs whose moments follow from orthogonality (Eq. 1 with Gauss-Legendre
nodes); library: numpy's FFT for the angular DFT; invariants: 90/180 degree
rotation, mirror (conjugation, Sec. 2 Z_{n,-m} = conj Z_nm), Neumann factor
(Eq. 14-15); brute force: hand-enumerated bilinear weights.
"""

import numpy as np
import pytest

from oracle import grid, moments, resample, zernike
from paper_2304_14492_gb300 import synth


def test_radial_quadrature_closed_forms():
    for n_rho in (1, 7, 32):
        rho, wr = grid.radial_nodes(n_rho, "midpoint")
        assert abs(wr.sum() - 0.5) <= 1e-15                  # integral of rho
        assert abs(rho[0] - 0.5 / n_rho) <= 1e-16 and abs(rho[-1] - 1 + 0.5 / n_rho) <= 1e-15
    for n in (1, 5, 40):
        rho, wr = grid.radial_nodes(n, "gauss")
        for k in range(0, 2 * n - 1):                      # degree k+1 <= 2n-1 exact
            assert abs(np.sum(wr * rho ** k) - 1.0 / (k + 2)) <= 1e-14
    th = grid.angles(8)
    assert np.allclose(th, np.arange(8) * np.pi / 4)
    assert grid.default_geometry(2160, 3840) == (1919.5, 1079.5, 1080.0)


def test_bilinear_hand_enumerated():
    img = np.arange(16, dtype=np.float64).reshape(4, 4) ** 1.5
    # point (X, Y) = (1.25, 2.5): neighbours (1,2) (2,2) (1,3) (2,3)
    want = 0.75 * 0.5 * img[2, 1] + 0.25 * 0.5 * img[2, 2] + 0.75 * 0.5 * img[3, 1] + 0.25 * 0.5 * img[3, 2]
    assert abs(resample.bilinear(img, 1.25, 2.5) - want) <= 1e-12
    # integer coordinates return the pixel
    assert resample.bilinear(img, 3.0, 1.0) == img[1, 3]
    # right/bottom edge: neighbour at x = 4 is outside -> zero
    assert abs(resample.bilinear(img, 3.5, 0.0) - 0.5 * img[0, 3]) <= 1e-12
    # left edge: X = -0.25 -> 0.75 * img[., 0] (x = -1 is outside)
    assert abs(resample.bilinear(img, -0.25, 2.0) - 0.75 * img[2, 0]) <= 1e-12
    assert resample.bilinear(img, -1.0, 2.0) == 0.0
    assert resample.bilinear(img, 1.0, 7.0) == 0.0


def test_bilinear_reproduces_linear_ramp():
    h, w = 9, 13
    y, x = np.mgrid[0:h, 0:w]
    img = 0.3 * x - 1.7 * y + 2.0
    rng = np.random.default_rng(1)
    X = rng.uniform(0, w - 1, 200)
    Y = rng.uniform(0, h - 1, 200)
    assert np.max(np.abs(resample.bilinear(img, X, Y) - (0.3 * X - 1.7 * Y + 2.0))) <= 1e-12


def test_constant_image_resamples_to_one():
    img = np.ones((64, 48))
    rho, _ = grid.radial_nodes(24, "midpoint")             # N_rho <= min(H, W) / 2
    f = resample.polar_resample(img, rho, 64)
    assert np.max(np.abs(f - 1.0)) <= 1e-14


def test_polar_resample_rotation_is_index_shift():
    img = synth.uniform_image(32, 32, workload=99, index=0).astype(np.float64)
    rho, _ = grid.radial_nodes(16, "midpoint")
    f = resample.polar_resample(img, rho, 64)
    f90 = resample.polar_resample(np.rot90(img), rho, 64)
    assert np.max(np.abs(f90 - np.roll(f, 16, axis=1))) <= 1e-12


def test_angular_dft_vs_numpy_fft():
    rng = np.random.default_rng(5)
    fhat = rng.standard_normal((7, 64))
    F = moments.angular_dft(fhat, 20)
    ref = np.fft.rfft(fhat, axis=1)[:, :21]
    assert np.max(np.abs(F - ref)) <= 1e-12


def test_constant_image_moments():
    img = np.ones((64, 64))
    Z = moments.moments(img, 20, 32, 64)
    pairs = zernike.index_pairs(20)
    assert abs(Z[0] - 1.0) <= 1e-14                       # Z_00 = 1
    for row, (n, m) in enumerate(pairs):
        if m > 0:
            assert abs(Z[row]) <= 1e-13                    # no angular content
    # Z_{n>0,0} vanishes only up to the midpoint rule's error ...
    assert max(abs(Z[r]) for r, (n, m) in enumerate(pairs) if m == 0 and n > 0) > 1e-8
    # ... and exactly on Gauss-Legendre nodes (whose outer node reaches
    # rho ~ 0.999, so the disk is kept one pixel inside the image)
    ZG = moments.moments(img, 20, 24, 64, grid="gauss", geometry=(31.5, 31.5, 30.0))
    assert abs(ZG[0] - 1.0) <= 1e-13
    assert np.max(np.abs(ZG[1:])) <= 1e-12


@pytest.mark.parametrize("np_,mp_", [(0, 0), (4, 2), (7, 3), (12, 12), (20, 6)])
def test_polar_zernike_input_closed_form(np_, mp_):
    # f_hat = R_{n'm'}(rho) cos(m' theta) -> Z_nm = delta delta eps_m'/2;
    # f_hat = R_{n'm'}(rho) sin(m' theta) -> Z_nm = -j/2 delta delta (m' > 0).
    n_max, n_theta = 24, 64
    n_rho = n_max + 1
    rho, _ = grid.radial_nodes(n_rho, "gauss")
    th = grid.angles(n_theta)
    R = zernike.zrp_table(np_, rho)[zernike.moment_index(np_, mp_)]
    pairs = zernike.index_pairs(n_max)
    target = zernike.moment_index(np_, mp_)
    Zc = moments.moments_polar(R[:, None] * np.cos(mp_ * th)[None, :], n_max, "gauss")
    want = np.zeros(len(pairs), complex)
    want[target] = 1.0 if mp_ == 0 else 0.5
    assert np.max(np.abs(Zc - want)) <= 1e-13
    if mp_ > 0:
        Zs = moments.moments_polar(R[:, None] * np.sin(mp_ * th)[None, :], n_max, "gauss")
        want = np.zeros(len(pairs), complex)
        want[target] = -0.5j
        assert np.max(np.abs(Zs - want)) <= 1e-13


def test_rotation_and_mirror_invariants():
    img = synth.uniform_image(64, 64, workload=0, index=0).astype(np.float64)
    n_max = 20
    pairs = zernike.index_pairs(n_max)
    ms = np.array([m for _, m in pairs])
    Z = moments.moments(img, n_max, 32, 64)
    Z90 = moments.moments(np.rot90(img), n_max, 32, 64)
    Z180 = moments.moments(np.rot90(img, 2), n_max, 32, 64)
    Zm = moments.moments(np.flipud(img), n_max, 32, 64)
    assert np.max(np.abs(Z90 - (-1j) ** ms * Z)) <= 1e-13     # counter-clockwise 90 deg
    assert np.max(np.abs(Z180 - (-1.0) ** ms * Z)) <= 1e-13
    assert np.max(np.abs(np.abs(Z90) - np.abs(Z))) <= 1e-13   # |Z| invariant
    assert np.max(np.abs(Zm - np.conj(Z))) <= 1e-13           # mirror in y


def test_neumann_division():
    img = synth.uniform_image(32, 32, workload=7, index=1).astype(np.float64)
    Z = moments.moments(img, 9, 16, 32)
    ZN = moments.moments(img, 9, 16, 32, neumann=True)
    for row, (n, m) in enumerate(zernike.index_pairs(9)):
        assert ZN[row] == Z[row] / (2.0 if m == 0 else 1.0)


def test_non_square_geometry_and_mirror_x():
    # a non-square image: mirror in x gives Z_nm -> (-1)^m conj(Z_nm)
    img = synth.uniform_image(24, 40, workload=8, index=0).astype(np.float64)
    ms = np.array([m for _, m in zernike.index_pairs(10)])
    Z = moments.moments(img, 10, 12, 32)
    Zx = moments.moments(np.fliplr(img), 10, 12, 32)
    assert np.max(np.abs(Zx - (-1.0) ** ms * np.conj(Z))) <= 1e-13
