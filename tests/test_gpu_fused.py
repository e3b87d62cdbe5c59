"""GPU parity of the fused resampling + ring FFT kernel (Sec. 2.5 and Eq. 1 in
one pass, polar samples kept on chip).

The fused kernel performs the same float operations as the two-pass path (the
resampler writes the polar samples, the ring-FFT kernel reads them back), so
its moments and its optional polar samples must equal that path's bit for bit;
both are also held to the oracle at 1e-4 * max|Z|.  Geometries cover disks
inside, across and beyond the image edges, ragged ring counts, every angle
count the warp FFT takes (64 .. 2048), both radial rules, the three
precisions, mixed batches and a geometry too large for the stage buffers.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grid, moments as om, resample  # noqa: E402
from paper_2304_14492_gb300 import native as zm, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL_Z = 1e-4
PRECS = {"fp32": zm.ZM_PREC_FP32, "bf16x3": zm.ZM_PREC_BF16X3, "fp16x3": zm.ZM_PREC_FP16X3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2304_14492_gb300.build import build
    build()
    zm.lib()


@pytest.fixture(autouse=True)
def _fused(monkeypatch):
    # plans made in these tests fuse wherever the geometry fits, whatever
    # their size (the library's automatic choice fuses small grids only)
    monkeypatch.setenv("ZM_FUSED", "1")
    monkeypatch.delenv("ZM_POLAR_DFT", raising=False)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def complex_of(out):
    o = out.double().cpu().numpy()
    return o[..., 0] + 1j * o[..., 1]


def fused_and_two_pass(plan, P, n_rho, n_theta, views, geometries=None):
    """(moments by zm_moments, moments by zm_moments_ex with polar samples,
    those samples, moments by resample + polar moments, the resampled samples,
    launches of the zm_moments call minus launches of the two-pass calls)."""
    B = len(views)
    a = torch.empty((B, P, 2), device=DEV)
    f2 = torch.full((B, n_rho, n_theta), float("nan"), device=DEV)
    # first calls build the per-geometry plans (the tile path launches its
    # planning kernels then); launches are counted on the second calls
    zm.zm_moments(plan, views, a, 0, geometries=geometries)
    zm.zm_resample(plan, views, f2, geometries=geometries)
    l0 = zm.zm_launch_count()
    zm.zm_moments(plan, views, a, 0, geometries=geometries)
    launches = zm.zm_launch_count() - l0
    a_ex = torch.empty((B, P, 2), device=DEV)
    f_ex = torch.full((B, n_rho, n_theta), float("nan"), device=DEV)
    zm.zm_moments_ex(plan, views, a_ex, f_ex, 0, geometries=geometries)
    f2.fill_(float("nan"))
    l0 = zm.zm_launch_count()
    zm.zm_resample(plan, views, f2, geometries=geometries)
    b = torch.empty((B, P, 2), device=DEV)
    zm.zm_moments_polar(plan, f2, B, b, 0)
    launches -= zm.zm_launch_count() - l0
    torch.cuda.synchronize()
    zm.zm_plan_status(plan)                      # no stencil outside its staged rows
    return a, a_ex, f_ex, b, f2, launches


CASES = [
    # shape, batch, n_max, n_rho, n_theta, geometry, grid flag
    ((64, 64), 1, 20, 32, 64, None, 0),                       # the small parity workload
    ((512, 512), 3, 50, 256, 256, None, 0),                   # blob frames, several images
    ((300, 200), 2, 30, 100, 512, (60.5, 250.0, 55.0), 0),    # off-centre disk
    ((40, 36), 1, 12, 25, 128, (18.0, 20.0, 60.0), 0),        # disk larger than the image, ragged rings
    ((256, 256), 1, 30, 64, 2048, None, 0),                   # 2048 angles
    ((128, 96), 2, 40, 47, 1024, (47.25, 63.75, 47.9), zm.ZM_GRID_GAUSS),
    ((96, 128), 1, 9, 200, 128, (-10.0, 40.0, 70.0), 0),      # centre left of the image
]


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("shape,B,n_max,n_rho,n_theta,geometry,gflag", CASES)
def test_fused_equals_two_pass_and_oracle(prec, shape, B, n_max, n_rho, n_theta, geometry, gflag):
    imgs = [synth.blob_image(shape[0], shape[1], 8, workload=21, index=j) for j in range(B)]
    views = [dev(i) for i in imgs]
    geos = [geometry] * B if geometry else None
    P = zm.zm_num_moments(n_max)
    plan = zm.zm_plan(n_max, n_rho, n_theta, PRECS[prec] | gflag)
    try:
        a, a_ex, f_ex, b, f2, launches = fused_and_two_pass(plan, P, n_rho, n_theta, views, geos)
    finally:
        zm.zm_plan_destroy(plan)
    # the fused kernel took the run: one launch where the two-pass path
    # launches the resampler and the ring FFT
    assert launches == -1, launches
    assert torch.equal(f_ex, f2), "polar samples differ from the resampler's"
    assert torch.equal(a, b), "fused moments differ from the two-pass moments"
    assert torch.equal(a, a_ex)
    Z = complex_of(a)
    for j in range(B):
        ref = om.moments(imgs[j].astype(np.float64), n_max, n_rho, n_theta,
                         grid="gauss" if gflag else "midpoint", geometry=geometry)
        assert np.max(np.abs(Z[j] - ref)) <= TOL_Z * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_fused_4k_frames(prec):
    """Two 4K frames (3840x2160, n_max 100, 1024 x 1024): fused = two-pass bit
    for bit, and frame 0's samples on sampled rings equal the oracle's."""
    imgs = [synth.blob_image(2160, 3840, 32, workload=2, index=j) for j in range(2)]
    views = [dev(i) for i in imgs]
    P = zm.zm_num_moments(100)
    plan = zm.zm_plan(100, 1024, 1024, PRECS[prec])
    try:
        a, a_ex, f_ex, b, f2, launches = fused_and_two_pass(plan, P, 1024, 1024, views)
    finally:
        zm.zm_plan_destroy(plan)
    assert launches == -1
    assert torch.equal(f_ex, f2)
    assert torch.equal(a, b)
    rings = np.array([0, 1, 15, 16, 17, 511, 512, 1000, 1022, 1023])
    rho, _ = grid.radial_nodes(1024)
    ref = resample.polar_resample(imgs[0].astype(np.float64), rho[rings], 1024)
    got = f_ex[0].double().cpu().numpy()[rings]
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_mixed_batch_runs():
    """A batch whose runs take different paths (fused, fused with another
    geometry, width not a multiple of 4 -> gather kernel) gives each image the
    moments it gets alone."""
    n_max, n_rho, n_theta = 24, 48, 128
    P = zm.zm_num_moments(n_max)
    shapes = [(96, 96), (96, 96), (96, 98), (96, 96)]
    geos = [None, (40.0, 50.0, 45.0), None, None]
    imgs = [synth.blob_image(h, w, 6, workload=22, index=j) for j, (h, w) in enumerate(shapes)]
    views = [dev(i) for i in imgs]
    plan = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_BF16X3)
    try:
        out = torch.empty((4, P, 2), device=DEV)
        zm.zm_moments(plan, views, out, 0, geometries=geos)
        alone = []
        for j in range(4):
            o = torch.empty((1, P, 2), device=DEV)
            zm.zm_moments(plan, [views[j]], o, 0, geometries=[geos[j]])
            alone.append(o)
        torch.cuda.synchronize()
        zm.zm_plan_status(plan)
    finally:
        zm.zm_plan_destroy(plan)
    Z = complex_of(out)
    for j in range(4):
        ref = om.moments(imgs[j].astype(np.float64), n_max, n_rho, n_theta, geometry=geos[j])
        assert np.max(np.abs(Z[j] - ref)) <= TOL_Z * np.max(np.abs(ref))
        # the projection accumulates the same columns in another batch: equal to rounding
        assert np.max(np.abs(Z[j] - complex_of(alone[j])[0])) <= 1e-6 * np.max(np.abs(ref))


def test_geometry_too_large_for_the_stage_buffers():
    """64 angles on a 2048 x 2048 frame: a 16-angle slot is a quarter of a
    ring of radius 1024, more rows than a stage holds; the batch falls back to
    the two-pass path and stays right."""
    img = synth.blob_image(2048, 2048, 8, workload=23, index=0)
    n_max, n_rho, n_theta = 20, 1024, 64
    P = zm.zm_num_moments(n_max)
    plan = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_FP32)
    try:
        out = torch.empty((1, P, 2), device=DEV)
        l0 = zm.zm_launch_count()
        zm.zm_moments(plan, [dev(img)], out, 0)
        launches = zm.zm_launch_count() - l0
        torch.cuda.synchronize()
    finally:
        zm.zm_plan_destroy(plan)
    assert launches >= 4          # tile resampler + ring FFT + projection + reduce
    ref = om.moments(img.astype(np.float64), n_max, n_rho, n_theta)
    Z = complex_of(out)[0]
    assert np.max(np.abs(Z - ref)) <= TOL_Z * np.max(np.abs(ref))


def test_automatic_choice_fuses_small_grids_only(monkeypatch):
    """Without ZM_FUSED a plan fuses up to 2^17 polar samples per image and
    resamples larger grids by tiles first; the moments are the same."""
    monkeypatch.delenv("ZM_FUSED")
    counts = {}
    for shape, n_max, n_rho, n_theta in (((512, 512), 50, 256, 256), ((1024, 1024), 60, 512, 512)):
        img = dev(synth.blob_image(shape[0], shape[1], 8, workload=25, index=0))
        P = zm.zm_num_moments(n_max)
        plan = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_BF16X3)
        try:
            a, _, _, b, _, launches = fused_and_two_pass(plan, P, n_rho, n_theta, [img])
        finally:
            zm.zm_plan_destroy(plan)
        assert torch.equal(a, b)
        counts[n_rho * n_theta] = launches
    assert counts[256 * 256] == -1          # fused: one launch where the two-pass path takes two
    assert counts[512 * 512] == 0           # 2^18 samples: the tile path
