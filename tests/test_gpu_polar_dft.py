"""GPU parity of the tensor-core DFT from polar samples: the angular sums of
Eq. 1, F_m(rho_i) = sum_k f_ik e^{-j m theta_k} for m <= n_max, as a split
bf16 product of the samples with the DFT matrix (FP32 accumulation), written
as the blocked projection's operand blocks.  bf16x3 plans made with
ZM_POLAR_DFT=1 take it for polar input (zm_moments_polar, and the tile path's
resampled samples); without it they keep the radix ring FFT.

Bars: the moments against the FP64 oracle at 2e-5 * max|Z| (the split forms'
bar) and against the ring-FFT path at the same bar, while differing from it
(the switch changes the arithmetic); against a CPU emulation of the kernel's
split to FP32 rounding; ring counts that leave a 128-ring tile partly or
wholly past the operand blocks, one stage (32 angles) and 64 stages, n_max 0
and 127, and the inputs it hands back to the ring FFT (an unaligned polar
buffer, n_max 128).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grid, moments as om, resample, zernike  # noqa: E402
from paper_2304_14492_gb300 import native as zm, synth  # noqa: E402
from splitmath import dft_split_spectra, split_moments  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL_SPLIT = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2304_14492_gb300.build import build
    build()
    zm.lib()


def complex_of(out):
    o = out.double().cpu().numpy()
    return o[..., 0] + 1j * o[..., 1]


def polar_samples(imgs, n_rho, n_theta):
    """The oracle's FP64 polar samples (Sec. 2.5) of each image, [B, N_rho, N_theta]."""
    rho, _ = grid.radial_nodes(n_rho)
    return np.stack([resample.polar_resample(i.astype(np.float64), rho, n_theta,
                                             grid.default_geometry(*i.shape)) for i in imgs])


def polar_moments(monkeypatch, mode, n_max, fh, offset=0):
    """zm_moments_polar on the samples fh (a float32 CUDA copy starting
    `offset` floats into its buffer) with ZM_POLAR_DFT=mode (unset for None)."""
    if mode is None:
        monkeypatch.delenv("ZM_POLAR_DFT", raising=False)
    else:
        monkeypatch.setenv("ZM_POLAR_DFT", mode)
    B, n_rho, n_theta = fh.shape
    buf = torch.zeros(offset + fh.size, device=DEV)
    buf[offset:] = torch.from_numpy(fh.astype(np.float32).ravel()).to(DEV)
    view = buf[offset:].view(B, n_rho, n_theta)
    plan = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_BF16X3)
    try:
        out = torch.full((B, zm.zm_num_moments(n_max), 2), float("nan"), device=DEV)
        zm.zm_moments_polar(plan, view, B, out, 0)
        torch.cuda.synchronize()
        zm.zm_plan_status(plan)                  # no bounded wait gave up
    finally:
        zm.zm_plan_destroy(plan)
    return complex_of(out)


CASES = [
    # image shape, batch, n_max, n_rho, n_theta
    ((64, 64), 1, 20, 32, 64),           # one tile, rings 32-127 past the blocks (one chunk)
    ((512, 512), 3, 50, 256, 256),       # two tiles
    ((300, 300), 2, 30, 100, 512),       # ragged rings: tile 0 rings 100-127 zero
    ((256, 256), 2, 127, 200, 256),      # 256 accumulator columns; second tile half past the rings
    ((128, 128), 2, 0, 64, 32),          # one order, one stage (fewer stages than slots)
    ((256, 256), 1, 40, 128, 2048),      # 64 stages
]


@pytest.mark.parametrize("shape,B,n_max,n_rho,n_theta", CASES)
def test_polar_dft_matches_oracle_and_ring_fft(monkeypatch, shape, B, n_max, n_rho, n_theta):
    imgs = [synth.blob_image(shape[0], shape[1], 8, workload=45, index=j) for j in range(B)]
    fh = polar_samples(imgs, n_rho, n_theta)
    Z = polar_moments(monkeypatch, "1", n_max, fh)
    Zf = polar_moments(monkeypatch, None, n_max, fh)          # off by default: the ring FFT
    assert not np.array_equal(Z, Zf), "the tensor-core DFT did not run"
    for j in range(B):
        ref = om.moments(imgs[j].astype(np.float64), n_max, n_rho, n_theta)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(Z[j] - ref)) <= TOL_SPLIT * scale, j
        assert np.max(np.abs(Z[j] - Zf[j])) <= TOL_SPLIT * scale, j


def test_polar_dft_hands_back_what_it_cannot_take(monkeypatch):
    """A polar buffer 8 bytes off a 16-byte boundary, and n_max = 128 (more
    accumulator columns than TMEM holds), take the ring FFT: equal to the
    result without the variable bit for bit."""
    img = synth.blob_image(256, 256, 8, workload=46, index=0)
    for n_max, n_rho, n_theta, off in ((30, 128, 256, 2), (128, 64, 512, 0)):
        fh = polar_samples([img], n_rho, n_theta)
        Z = polar_moments(monkeypatch, "1", n_max, fh, offset=off)
        Zf = polar_moments(monkeypatch, None, n_max, fh, offset=off)
        assert np.array_equal(Z, Zf), (n_max, off)


def test_polar_dft_equals_emulated_split(monkeypatch):
    """The kernel's moments = CPU emulation of its arithmetic on the same FP32
    samples (split DFT, FP32 spectra, split projection) to the FP32 rounding
    of both accumulations: 2^-19 (S_nm + S'_nm), S'_nm = sum_i |a_i| sum_k |f_ik|."""
    n_max, n_rho, n_theta = 50, 256, 512
    imgs = [synth.blob_image(512, 512, 8, workload=47, index=j) for j in range(2)]
    fh = polar_samples(imgs, n_rho, n_theta).astype(np.float32).astype(np.float64)
    Z = polar_moments(monkeypatch, "1", n_max, fh)
    rho, wr = grid.radial_nodes(n_rho)
    T = zernike.zrp_table(n_max, rho)
    pairs = zernike.index_pairs(n_max)
    a = np.array([(n + 1) / np.pi * wr * (2 * np.pi / n_theta) * T[r] for r, (n, m) in enumerate(pairs)])
    ms = [m for _, m in pairs]
    for b in range(2):
        F = dft_split_spectra(fh[b], n_max, 8).astype(np.complex64).astype(np.complex128)
        f = F[:, ms].T
        emu = split_moments(a, f, 8)
        S = np.sum(np.abs(a) * np.abs(f), axis=1) + np.abs(a) @ np.sum(np.abs(fh[b]), axis=1)
        assert np.all(np.abs(Z[b] - emu) <= 2.0 ** -19 * S + 2.0 ** -30 * np.max(S)), b
