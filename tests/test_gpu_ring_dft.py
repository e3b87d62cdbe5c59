"""GPU parity of the tensor-core DFT kernel: bilinear polar resampling (Sec.
2.5) with the angular sums of Eq. 1 computed as a product of the samples with
the DFT matrix on the tensor cores (bf16 hi + lo split of both operands, FP32
accumulation), feeding the blocked tensor-core projection.

Bars: the moments against the FP64 oracle at 2e-5 * max|Z| (the split forms'
bar); against a CPU emulation of the kernel's own split, on the GPU's own FP32
polar samples, to FP32 rounding (so that a weaker split cannot pass); the
kernel taking the run (one launch fewer than the tile resampler + ring FFT);
geometries with one band, an unpaired middle band, disks across and beyond the
image, ragged ring counts, n_max 0 and 127 (the widest accumulator), 2048
angles, batches over one launch's image limit, mixed batches, and geometries
the kernel hands back to the other paths.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grid, moments as om, zernike  # noqa: E402
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def complex_of(out):
    o = out.double().cpu().numpy()
    return o[..., 0] + 1j * o[..., 1]


def moments(monkeypatch, mode, n_max, n_rho, n_theta, views, geometries=None, fused="0"):
    """Moments of a bf16 plan made with ZM_RING_DFT=mode (unset for None), and
    the launches of a second call (the first builds the per-geometry plans)."""
    if mode is None:
        monkeypatch.delenv("ZM_RING_DFT", raising=False)
    else:
        monkeypatch.setenv("ZM_RING_DFT", mode)
    monkeypatch.setenv("ZM_FUSED", fused)
    plan = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_BF16X3)
    try:
        out = torch.empty((len(views), zm.zm_num_moments(n_max), 2), device=DEV)
        zm.zm_moments(plan, views, out, 0, geometries=geometries)
        out.fill_(float("nan"))
        l0 = zm.zm_launch_count()
        zm.zm_moments(plan, views, out, 0, geometries=geometries)
        launches = zm.zm_launch_count() - l0
        torch.cuda.synchronize()
        zm.zm_plan_status(plan)                  # no bounded wait gave up
    finally:
        zm.zm_plan_destroy(plan)
    return complex_of(out), launches


CASES = [
    # shape, batch, n_max, n_rho, n_theta, geometry
    ((64, 64), 1, 20, 32, 64, None),                          # one band, no partner
    ((512, 512), 3, 50, 256, 256, None),                      # 4 bands: 2 pairs
    ((300, 200), 2, 30, 100, 512, (60.5, 250.0, 55.0)),       # off-centre disk across the edge, ragged rings
    ((40, 36), 1, 12, 25, 128, (18.0, 20.0, 60.0)),           # disk larger than the image
    ((256, 256), 2, 127, 320, 256, None),                     # 256 accumulator columns; 5 bands (middle unpaired)
    ((96, 128), 2, 0, 200, 128, (-10.0, 40.0, 70.0)),         # one order; centre left of the image
    ((128, 128), 1, 40, 64, 2048, None),                      # 2048 angles: 128 stages
    ((128, 96), 2, 40, 47, 1024, (47.25, 63.75, 47.9)),       # ragged rings, fractional centre
]


@pytest.mark.parametrize("shape,B,n_max,n_rho,n_theta,geometry", CASES)
def test_dft_kernel_matches_oracle(monkeypatch, shape, B, n_max, n_rho, n_theta, geometry):
    imgs = [synth.blob_image(shape[0], shape[1], 8, workload=40, index=j) for j in range(B)]
    views = [dev(i) for i in imgs]
    geos = [geometry] * B if geometry else None
    Z, l_dft = moments(monkeypatch, "1", n_max, n_rho, n_theta, views, geos)
    Zt, l_tile = moments(monkeypatch, "0", n_max, n_rho, n_theta, views, geos)
    assert l_dft == l_tile - 1, (l_dft, l_tile)     # one kernel where the tile path runs two
    for j in range(B):
        ref = om.moments(imgs[j].astype(np.float64), n_max, n_rho, n_theta, geometry=geometry)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(Z[j] - ref)) <= TOL_SPLIT * scale, j
        assert np.max(np.abs(Zt[j] - ref)) <= TOL_SPLIT * scale, j


def weights(n_max, n_rho, n_theta):
    """a_nm,i = (n+1)/pi * w_i * 2pi/N_theta * R_nm(rho_i), FP64 (Eq. 1)."""
    rho, wr = grid.radial_nodes(n_rho)
    T = zernike.zrp_table(n_max, rho)
    pairs = zernike.index_pairs(n_max)
    a = np.array([(n + 1) / np.pi * wr * (2 * np.pi / n_theta) * T[r] for r, (n, m) in enumerate(pairs)])
    return a, [m for _, m in pairs]


@pytest.mark.parametrize("shape,n_max,n_rho,n_theta,geometry", [
    ((512, 512), 50, 256, 256, None),
    ((300, 200), 30, 100, 512, (60.5, 250.0, 55.0)),
])
def test_dft_kernel_equals_emulated_split(monkeypatch, shape, n_max, n_rho, n_theta, geometry):
    """Moments of the kernel = CPU emulation of its arithmetic on the GPU's own
    FP32 polar samples: split DFT (f_hi w_hi + f_hi w_lo + f_lo w_hi), FP32
    spectra, split projection; to the FP32 rounding of both accumulations,
    2^-19 (S_nm + S'_nm) with S'_nm = sum_i |a_i| sum_k |f_ik|."""
    B = 2
    imgs = [synth.blob_image(shape[0], shape[1], 8, workload=41, index=j) for j in range(B)]
    views = [dev(i) for i in imgs]
    geos = [geometry] * B if geometry else None
    Z, _ = moments(monkeypatch, "1", n_max, n_rho, n_theta, views, geos)
    plan = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_BF16X3)
    try:
        fh = torch.empty((B, n_rho, n_theta), device=DEV)
        zm.zm_resample(plan, views, fh, geometries=geos)
        torch.cuda.synchronize()
        fh = fh.double().cpu().numpy()
    finally:
        zm.zm_plan_destroy(plan)
    a, ms = weights(n_max, n_rho, n_theta)
    for b in range(B):
        F = dft_split_spectra(fh[b], n_max, 8).astype(np.complex64).astype(np.complex128)
        f = F[:, ms].T                                       # [P, N_rho]
        emu = split_moments(a, f, 8)
        L1 = np.sum(np.abs(fh[b]), axis=1)
        S = np.sum(np.abs(a) * np.abs(f), axis=1) + np.abs(a) @ L1
        assert np.all(np.abs(Z[b] - emu) <= 2.0 ** -19 * S + 2.0 ** -30 * np.max(S)), b


def test_dft_kernel_4k_frames(monkeypatch):
    """Two 4K frames (3840x2160, disk d=2160, n_max 100, 1024 x 1024) against
    the oracle at the split bar; without ZM_RING_DFT the plan keeps the tile
    path."""
    imgs = [synth.blob_image(2160, 3840, 32, workload=2, index=j) for j in range(2)]
    views = [dev(i) for i in imgs]
    Z, l_dft = moments(monkeypatch, "1", 100, 1024, 1024, views)
    assert l_dft == 2                              # the kernel and the projection
    for j in range(2):
        ref = om.moments(imgs[j].astype(np.float64), 100, 1024, 1024)
        assert np.max(np.abs(Z[j] - ref)) <= TOL_SPLIT * np.max(np.abs(ref)), j
    # off by default: a plan made without the variable takes the tile path
    Zd, l_default = moments(monkeypatch, None, 100, 1024, 1024, views)
    assert l_default == 3                          # tile resampler, ring FFT, projection
    assert np.max(np.abs(Zd - Z)) <= TOL_SPLIT * np.max(np.abs(Z))


def test_dft_kernel_over_one_launch_of_images(monkeypatch):
    """130 images (one launch takes 128): every image gets the moments it gets
    alone."""
    n_max, n_rho, n_theta = 16, 32, 64
    imgs = [synth.blob_image(64, 64, 4, workload=42, index=j) for j in range(130)]
    views = [dev(i) for i in imgs]
    Z, launches = moments(monkeypatch, "1", n_max, n_rho, n_theta, views)
    assert launches == 3                           # two kernel launches and the projection
    for j in (0, 127, 128, 129):
        ref = om.moments(imgs[j].astype(np.float64), n_max, n_rho, n_theta)
        assert np.max(np.abs(Z[j] - ref)) <= TOL_SPLIT * np.max(np.abs(ref)), j


def test_dft_kernel_in_a_mixed_batch(monkeypatch):
    """Runs of two geometries and an image whose width is not a multiple of 4
    (the gather kernel takes it): each image as alone."""
    n_max, n_rho, n_theta = 24, 96, 128
    shapes = [(160, 160), (160, 160), (160, 162), (160, 160)]
    geos = [None, (70.0, 80.0, 75.0), None, None]
    imgs = [synth.blob_image(h, w, 6, workload=43, index=j) for j, (h, w) in enumerate(shapes)]
    views = [dev(i) for i in imgs]
    Z, _ = moments(monkeypatch, "1", n_max, n_rho, n_theta, views, geos)
    for j in range(4):
        ref = om.moments(imgs[j].astype(np.float64), n_max, n_rho, n_theta, geometry=geos[j])
        assert np.max(np.abs(Z[j] - ref)) <= TOL_SPLIT * np.max(np.abs(ref)), j


def test_geometries_the_dft_kernel_hands_back(monkeypatch):
    """A stage that the buffers cannot hold (64 angles on a 2048 x 2048 frame:
    a 16-angle stage is a quarter of the outer rings) and n_max = 130 (more
    accumulator columns than TMEM holds) take the tile path: the same
    launches as with the kernel switched off, and moments at the bar."""
    for shape, n_max, n_rho, n_theta in (((2048, 2048), 20, 1024, 64), ((128, 128), 130, 64, 512)):
        img = synth.blob_image(shape[0], shape[1], 8, workload=44, index=0)
        views = [dev(img)]
        Z, l_on = moments(monkeypatch, "1", n_max, n_rho, n_theta, views)
        _, l_off = moments(monkeypatch, "0", n_max, n_rho, n_theta, views)
        assert l_on == l_off
        ref = om.moments(img.astype(np.float64), n_max, n_rho, n_theta)
        assert np.max(np.abs(Z[0] - ref)) <= TOL_SPLIT * np.max(np.abs(ref))
