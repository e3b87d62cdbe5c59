"""GPU parity: every step of the CUDA path against the FP64 oracle, through the
C ABI (run with -m gpu on a GB300).

Bars: the FP64 table of Eq. 7 within 1e-12 of the oracle's recurrence (and a
Gram matrix within 1e-10 of diag 1/(2(n+1)) on Gauss-Legendre nodes); FP32
moments within 1e-4 * max|Z| of the oracle (the stated tolerance); component
stages within bounds derived from FP32 rounding of their inputs.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grid, metrics, moments as om, reconstruct as orc, resample, zernike  # noqa: E402
from paper_2304_14492_gb300 import native as zm, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL_Z = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2304_14492_gb300.build import build
    build()
    zm.lib()


class Plan:
    def __init__(self, n_max, n_rho, n_theta, flags=0):
        self.h = zm.zm_plan(n_max, n_rho, n_theta, flags)
        self.n_max, self.n_rho, self.n_theta = n_max, n_rho, n_theta
        self.P = zm.zm_num_moments(n_max)
        self.grid = "gauss" if flags & zm.ZM_GRID_GAUSS else "midpoint"

    def __enter__(self):
        return self

    def __exit__(self, *a):
        zm.zm_plan_destroy(self.h)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def as_complex(out):
    o = out.double().cpu().numpy()
    return o[..., 0] + 1j * o[..., 1]


def gpu_moments(plan, imgs, flags=0, geometries=None):
    ts = [dev(i) for i in imgs]
    out = torch.empty((len(ts), plan.P, 2), device=DEV)
    zm.zm_moments(plan.h, ts, out, flags, geometries=geometries)
    torch.cuda.synchronize()
    return as_complex(out)


def oracle_moments(img, plan, neumann=False, geometry=None):
    return om.moments(np.asarray(img, np.float32).astype(np.float64), plan.n_max, plan.n_rho, plan.n_theta,
                      grid=plan.grid, neumann=neumann, geometry=geometry)


# ------------------------------------------------------------------ a1: Eq. 7 table
@pytest.mark.parametrize("n_max,n_rho,n_theta,flags", [
    (20, 32, 64, 0), (50, 256, 256, 0), (100, 1024, 1024, 0), (0, 1, 8, 0),
    (13, 37, 32, zm.ZM_GRID_GAUSS), (200, 202, 512, zm.ZM_GRID_GAUSS)])
def test_table_eq7_matches_recurrence(n_max, n_rho, n_theta, flags):
    with Plan(n_max, n_rho, n_theta, flags) as p:
        R = torch.empty((p.P, n_rho), device=DEV, dtype=torch.float64)
        rho = torch.empty(n_rho, device=DEV, dtype=torch.float64)
        wr = torch.empty(n_rho, device=DEV, dtype=torch.float64)
        zm.zm_plan_table(p.h, R)
        zm.zm_plan_nodes(p.h, rho, wr)
        torch.cuda.synchronize()
        R, rho, wr = R.cpu().numpy(), rho.cpu().numpy(), wr.cpu().numpy()
    rho_o, wr_o = grid.radial_nodes(n_rho, p.grid)
    assert np.max(np.abs(rho - rho_o)) <= 1e-14
    assert np.max(np.abs(wr - wr_o)) <= 1e-14 * max(1.0, np.max(np.abs(wr_o))) + 1e-16
    ref = zernike.zrp_table(n_max, rho_o)
    assert np.max(np.abs(R - ref)) <= 1e-12
    if flags & zm.ZM_GRID_GAUSS and n_rho >= n_max + 1:
        pairs = zernike.index_pairs(n_max)
        worst = 0.0
        for m in range(n_max + 1):
            rows = [r for r, (n, mm) in enumerate(pairs) if mm == m]
            ns = np.array([pairs[r][0] for r in rows])
            G = (R[rows] * wr) @ R[rows].T
            worst = max(worst, np.max(np.abs(G - np.diag(1.0 / (2.0 * (ns + 1))))))
        assert worst <= 1e-10, worst


# ------------------------------------------------------------------ a2: resampling
def gpu_resample(plan_args, imgs, geometries=None, views=None):
    n_max, n_rho, n_theta = plan_args
    with Plan(n_max, n_rho, n_theta) as p:
        f = torch.full((len(imgs), n_rho, n_theta), float("nan"), device=DEV)
        ts = views if views is not None else [dev(i) for i in imgs]
        zm.zm_resample(p.h, ts, f, geometries=geometries)
        torch.cuda.synchronize()
    return f.double().cpu().numpy()


@pytest.mark.parametrize("shape,n_rho,n_theta,geometry", [
    ((64, 64), 32, 64, None), ((45, 70), 21, 32, None), ((50, 40), 17, 64, (10.25, 30.5, 28.0)),
    ((40, 36), 25, 128, (18.0, 20.0, 60.0)),          # disk larger than the image
    ((300, 200), 100, 512, (60.5, 250.0, 55.0)),      # off-centre disk
    ((8, 8), 3, 8, None), ((1, 1), 2, 8, None)])
def test_resample_matches_oracle(shape, n_rho, n_theta, geometry):
    img = synth.uniform_image(*shape, workload=11, index=0)
    got = gpu_resample((4 if n_theta >= 16 else 3, n_rho, n_theta), [img], [geometry] if geometry else None)[0]
    rho, _ = grid.radial_nodes(n_rho)
    ref = resample.polar_resample(img.astype(np.float64), rho, n_theta, geometry)
    assert not np.isnan(got).any()
    assert np.max(np.abs(got - ref)) <= 2e-5


def test_resample_4k_frame():
    img = synth.blob_image(2160, 3840, 32, workload=2, index=0)
    got = gpu_resample((100, 1024, 1024), [img])[0]
    rho, _ = grid.radial_nodes(1024)
    ref = resample.polar_resample(img.astype(np.float64), rho, 1024)
    assert not np.isnan(got).any()
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_resample_strided_and_unaligned_views():
    # a pitch-100 view (16-byte aligned rows: tile path) and a view shifted by one
    # column (unaligned base: fused gather path) in one batch
    big = synth.uniform_image(80, 100, workload=12, index=0)
    t = dev(big)
    views = [t[4:68, 8:72], t[5:69, 9:73], t[4:68, 8:72]]
    imgs = [big[4:68, 8:72], big[5:69, 9:73], big[4:68, 8:72]]
    got = gpu_resample((4, 32, 64), imgs, views=views)
    rho, _ = grid.radial_nodes(32)
    for b in range(3):
        ref = resample.polar_resample(imgs[b].astype(np.float64), rho, 64)
        assert not np.isnan(got[b]).any()
        assert np.max(np.abs(got[b] - ref)) <= 2e-5


# ------------------------------------------------------------------ a3: ring spectra
@pytest.mark.parametrize("n_max,n_rho,n_theta", [(20, 32, 64), (3, 9, 8), (13, 37, 32), (100, 64, 1024),
                                                 (300, 16, 1024), (500, 8, 2048)])
def test_ring_spectra_match_direct_dft(n_max, n_rho, n_theta):
    img = synth.uniform_image(2 * n_rho + 3, 2 * n_rho + 1, workload=13, index=n_max)
    with Plan(n_max, n_rho, n_theta) as p:
        F = torch.empty((n_max + 1, 1, 2, n_rho), device=DEV)
        fh = torch.empty((1, n_rho, n_theta), device=DEV)
        zm.zm_ring_spectra(p.h, [dev(img)], F, fh)
        torch.cuda.synchronize()
    Fg = F[:, 0, 0, :].double().cpu().numpy() + 1j * F[:, 0, 1, :].double().cpu().numpy()   # [m][i]
    ref = om.angular_dft(fh[0].double().cpu().numpy(), n_max)                               # [i][m]
    assert np.max(np.abs(Fg.T - ref)) <= 2e-6 * np.max(np.abs(ref)) * np.log2(n_theta)


# ------------------------------------------------------------------ a3-a5 on polar input
@pytest.mark.parametrize("npr,mpr", [(0, 0), (6, 2), (11, 5), (24, 24), (30, 12)])
def test_polar_zernike_input_closed_form(npr, mpr):
    n_max, n_theta = 30, 64
    n_rho = n_max + 1
    rho, _ = grid.radial_nodes(n_rho, "gauss")
    th = grid.angles(n_theta)
    R = zernike.zrp_table(npr, rho)[zernike.moment_index(npr, mpr)]
    fc = R[:, None] * np.cos(mpr * th)[None, :]
    fs = R[:, None] * np.sin(mpr * th)[None, :]
    with Plan(n_max, n_rho, n_theta, zm.ZM_GRID_GAUSS) as p:
        fh = dev(np.stack([fc, fs]))
        out = torch.empty((2, p.P, 2), device=DEV)
        zm.zm_moments_polar(p.h, fh, 2, out)
        torch.cuda.synchronize()
        Z = as_complex(out)
    k = zernike.moment_index(npr, mpr)
    want = np.zeros(p.P, complex)
    want[k] = 1.0 if mpr == 0 else 0.5
    assert np.max(np.abs(Z[0] - want)) <= 1e-5
    if mpr > 0:
        want[k] = -0.5j
        assert np.max(np.abs(Z[1] - want)) <= 1e-5


def test_moments_polar_matches_oracle():
    rng = np.random.default_rng(3)
    n_max, n_rho, n_theta = 25, 40, 64
    fh = rng.random((3, n_rho, n_theta)).astype(np.float32)
    with Plan(n_max, n_rho, n_theta) as p:
        out = torch.empty((3, p.P, 2), device=DEV)
        zm.zm_moments_polar(p.h, dev(fh), 3, out, zm.ZM_NEUMANN)
        torch.cuda.synchronize()
        Z = as_complex(out)
    for b in range(3):
        ref = om.moments_polar(fh[b].astype(np.float64), n_max, neumann=True)
        assert metrics.rel_max_err(Z[b], ref) <= TOL_Z


# ------------------------------------------------------------------ a2-a5 end to end
@pytest.mark.parametrize("neumann", [False, True])
def test_moments_uniform_64(neumann):
    # 64x64 U[0,1] image, n_max 20, 32 x 64 grid
    img = synth.uniform_image(64, 64, workload=0, index=0)
    with Plan(20, 32, 64) as p:
        Z = gpu_moments(p, [img], zm.ZM_NEUMANN if neumann else 0)[0]
        ref = oracle_moments(img, p, neumann=neumann)
    assert metrics.rel_max_err(Z, ref) <= TOL_Z


def test_moments_blob_batch_512():
    # 16 blob images of 512x512, n_max 50, 256 x 256 grid
    imgs = [synth.blob_image(512, 512, 8, workload=1, index=b) for b in range(16)]
    with Plan(50, 256, 256) as p:
        Z = gpu_moments(p, imgs)
        for b in range(16):
            assert metrics.rel_max_err(Z[b], oracle_moments(imgs[b], p)) <= TOL_Z


def test_moments_ragged_and_uneven():
    # ragged ring blocks (N_rho = 37), odd n_max, N_theta = next pow2 >= 2 n_max + 2,
    # images of different sizes and geometries in one batch
    imgs = [synth.uniform_image(45, 70, workload=2, index=0), synth.uniform_image(33, 33, workload=2, index=1),
            synth.blob_image(90, 60, 3, workload=2, index=2)]
    geos = [None, (16.0, 16.0, 16.0), (20.5, 40.25, 35.0)]
    with Plan(13, 37, 32) as p:
        Z = gpu_moments(p, imgs, geometries=[g if g else (0, 0, -1) for g in geos])
        for b in range(3):
            assert metrics.rel_max_err(Z[b], oracle_moments(imgs[b], p, geometry=geos[b])) <= TOL_Z


def test_moments_mixed_alignment_batch():
    big = synth.blob_image(140, 150, 6, workload=14, index=0)
    t = dev(big)
    views = [t[0:128, 0:128], t[1:129, 3:131], t[6:134, 8:136]]
    imgs = [big[0:128, 0:128], big[1:129, 3:131], big[6:134, 8:136]]
    with Plan(30, 64, 64) as p:
        out = torch.empty((3, p.P, 2), device=DEV)
        zm.zm_moments(p.h, views, out)
        torch.cuda.synchronize()
        Z = as_complex(out)
        for b in range(3):
            assert metrics.rel_max_err(Z[b], oracle_moments(imgs[b], p)) <= TOL_Z


def test_moments_batch_spanning_launches_and_order_independence():
    imgs = [synth.uniform_image(16, 16, workload=4, index=b) for b in range(130)]
    with Plan(5, 8, 16) as p:
        Z = gpu_moments(p, imgs)
        alone = gpu_moments(p, [imgs[129]])[0]
        for b in (0, 64, 127, 128, 129):
            assert metrics.rel_max_err(Z[b], oracle_moments(imgs[b], p)) <= TOL_Z
    assert np.max(np.abs(alone - Z[129])) <= 1e-6 * np.max(np.abs(alone))


@pytest.mark.parametrize("n_max,n_rho,n_theta,shape", [(0, 1, 8, (4, 4)), (1, 2, 8, (1, 1)), (3, 5, 8, (8, 8)),
                                                        (127, 64, 256, (128, 128)), (511, 32, 1024, (64, 64)),
                                                        (1023, 8, 2048, (16, 16))])
def test_moments_edge_sizes(n_max, n_rho, n_theta, shape):
    img = synth.uniform_image(*shape, workload=5, index=n_max)
    with Plan(n_max, n_rho, n_theta) as p:
        Z = gpu_moments(p, [img])[0]
        ref = oracle_moments(img, p)
    assert metrics.rel_max_err(Z, ref) <= TOL_Z


def test_moments_gauss_grid_and_constant_image():
    img = np.ones((64, 64), np.float32)
    with Plan(20, 24, 64, zm.ZM_GRID_GAUSS) as p:
        Z = gpu_moments(p, [img], geometries=[(31.5, 31.5, 30.0)])[0]
    assert abs(Z[0] - 1.0) <= 1e-6
    assert np.max(np.abs(Z[1:])) <= 1e-6


def test_rotation_invariance_on_gpu():
    img = synth.blob_image(128, 128, 6, workload=6, index=0)
    with Plan(30, 64, 128) as p:
        Z = gpu_moments(p, [img, np.rot90(img).copy()])
    ms = np.array([m for _, m in zernike.index_pairs(30)])
    assert np.max(np.abs(Z[1] - (-1j) ** ms * Z[0])) <= 1e-5 * np.max(np.abs(Z[0]))


def test_deterministic():
    img = synth.blob_image(256, 256, 6, workload=7, index=0)
    with Plan(40, 128, 128) as p:
        a = gpu_moments(p, [img, img])
        b = gpu_moments(p, [img, img])
    assert np.array_equal(a, b)


# ------------------------------------------------------------------ a6: reconstruction
@pytest.mark.parametrize("neumann", [False, True])
@pytest.mark.parametrize("n_max,n_rho,n_theta", [(20, 32, 64), (13, 37, 32), (100, 128, 256), (0, 3, 8)])
def test_reconstruct_polar_matches_oracle(neumann, n_max, n_rho, n_theta):
    img = synth.uniform_image(2 * n_rho, 2 * n_rho, workload=8, index=n_max)
    with Plan(n_max, n_rho, n_theta) as p:
        Zref = oracle_moments(img, p)
        zin = dev(np.stack([Zref.real, Zref.imag], -1)[None])
        out = torch.empty((1, n_rho, n_theta), device=DEV)
        zm.zm_reconstruct(p.h, zin, 1, out, zm.ZM_NEUMANN if neumann else 0)
        torch.cuda.synchronize()
    ref = orc.reconstruct_polar(Zref.astype(np.complex64).astype(np.complex128), n_max, n_rho, n_theta,
                                neumann=neumann)
    assert np.max(np.abs(out[0].double().cpu().numpy() - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n_max,n_rho,n_theta", [(20, 32, 64), (13, 37, 32), (100, 256, 1024)])
def test_reconstruct_errors_fused_matches_separate_and_oracle(n_max, n_rho, n_theta):
    imgs = [synth.blob_image(2 * n_rho + 2, 2 * n_rho, 5, workload=15, index=b) for b in range(3)]
    with Plan(n_max, n_rho, n_theta) as p:
        out = torch.empty((3, p.P, 2), device=DEV)
        fh = torch.empty((3, n_rho, n_theta), device=DEV)
        zm.zm_moments_ex(p.h, [dev(i) for i in imgs], out, fh)
        rec = torch.empty((3, n_rho, n_theta), device=DEV)
        err_sep = torch.empty((3, 4), device=DEV, dtype=torch.float64)
        zm.zm_reconstruct(p.h, out, 3, rec, zm.ZM_NEUMANN)
        zm.zm_errors_polar(p.h, fh, rec, 3, err_sep)
        rec2 = torch.empty((3, n_rho, n_theta), device=DEV)
        err = torch.empty((3, 4), device=DEV, dtype=torch.float64)
        zm.zm_reconstruct_errors(p.h, out, 3, rec2, fh, err, zm.ZM_NEUMANN)
        err3 = torch.empty((3, 4), device=DEV, dtype=torch.float64)
        zm.zm_reconstruct_errors(p.h, out, 3, None, fh, err3, zm.ZM_NEUMANN)
        torch.cuda.synchronize()
        Z = as_complex(out)
    assert torch.equal(rec, rec2)
    e1, e2, e3 = err_sep.cpu().numpy(), err.cpu().numpy(), err3.cpu().numpy()
    assert np.array_equal(e2, e3)
    assert np.max(np.abs(e1 - e2) / np.abs(e1)) <= 1e-5
    f = fh.double().cpu().numpy()
    for b in range(3):
        r = orc.reconstruct_polar(Z[b], n_max, n_rho, n_theta, neumann=True)
        eps1 = np.sum((f[b] - r) ** 2) / np.sum(f[b] ** 2)
        eps = np.sum((f[b] - r) ** 2) / (f[b].max() ** 2 * f[b].size)
        assert abs(e2[b, 0] - eps1) <= 1e-4 * eps1 and abs(e2[b, 1] - eps) <= 1e-4 * eps
        assert e2[b, 3] == n_rho * n_theta


def test_reconstruct_cartesian_matches_oracle():
    h, w = 60, 75
    img = synth.blob_image(h, w, 4, workload=9, index=0)
    n_max, n_rho, n_theta = 24, 30, 64
    with Plan(n_max, n_rho, n_theta) as p:
        Zref = oracle_moments(img, p)
        zin = dev(np.stack([Zref.real, Zref.imag], -1)[None])
        canvas = torch.full((h, w), 7.0, device=DEV)
        polar = torch.empty((1, n_rho, n_theta), device=DEV)
        zm.zm_reconstruct_cartesian(p.h, zin, [canvas], polar, zm.ZM_NEUMANN)
        torch.cuda.synchronize()
    rho, _ = grid.radial_nodes(n_rho)
    fp = orc.reconstruct_polar(Zref, n_max, n_rho, n_theta, neumann=True)
    ref = orc.polar_to_cartesian(fp, rho, h, w)
    geo = grid.default_geometry(h, w)
    y, x = np.mgrid[0:h, 0:w]
    r_xy, _ = grid.pixel_to_polar(x, y, geo)
    sel = np.abs(r_xy - 1.0) > 1e-5
    got = canvas.double().cpu().numpy()
    assert np.max(np.abs(got[sel] - ref[sel])) <= 1e-4 * np.max(np.abs(ref))
    assert np.all(got[r_xy > 1.0 + 1e-5] == 0.0)


# ------------------------------------------------------------------ a7: errors and min-max
def test_errors_and_minmax_match_oracle():
    h, w = 70, 64
    f = synth.blob_image(h, w, 5, workload=10, index=0)
    g = f + synth.uniform_image(h, w, workload=10, index=1) * 0.1
    mask = metrics.disk_mask(h, w)
    with Plan(4, 8, 16) as p:
        out = torch.empty((1, 4), device=DEV, dtype=torch.float64)
        zm.zm_errors(p.h, [dev(f)], [dev(g)], out)
        mm = torch.empty((1, 2), device=DEV)
        zm.zm_disk_minmax(p.h, [dev(f)], mm)
        cv = dev(g)
        target = torch.tensor([[0.0, 255.0]], device=DEV)
        zm.zm_minmax_normalize(p.h, [cv], target)
        fr = torch.empty((1, 8, 16), device=DEV)
        fr2 = torch.empty((1, 8, 16), device=DEV)
        zm.zm_resample(p.h, [dev(f)], fr)
        zm.zm_resample(p.h, [dev(g)], fr2)
        outp = torch.empty((1, 4), device=DEV, dtype=torch.float64)
        zm.zm_errors_polar(p.h, fr, fr2, 1, outp)
        torch.cuda.synchronize()
    o = out[0].cpu().numpy()
    assert abs(o[0] - metrics.eps1(f, g, mask)) <= 1e-4 * metrics.eps1(f, g, mask)
    assert abs(o[1] - metrics.eps13(f, g, mask)) <= 1e-4 * metrics.eps13(f, g, mask)
    assert o[3] == mask.sum()
    m = mm[0].cpu().numpy()
    assert abs(m[0] - f[mask].min()) <= 1e-7 and abs(m[1] - f[mask].max()) <= 1e-7
    ref = metrics.minmax_normalize(g.astype(np.float64), 0.0, 255.0, mask)
    got = cv.double().cpu().numpy()
    assert np.max(np.abs(got[mask] - ref[mask])) <= 1e-3
    assert np.array_equal(got[~mask], g[~mask])
    a, b = fr[0].double().cpu().numpy(), fr2[0].double().cpu().numpy()
    op = outp[0].cpu().numpy()
    assert abs(op[0] - np.sum((a - b) ** 2) / np.sum(a ** 2)) <= 1e-4 * op[0]
    assert abs(op[1] - np.sum((a - b) ** 2) / (a.max() ** 2 * a.size)) <= 1e-4 * op[1]


# ------------------------------------------------------------------ argument errors
def test_argument_errors_on_gpu():
    with Plan(4, 8, 16) as p:
        x = dev(np.zeros((8, 8)))
        out = torch.empty((1, p.P, 2), device=DEV)
        with pytest.raises(zm.ZmError) as e:
            zm.zm_moments(p.h, [x], out, flags=0x80)
        assert e.value.status == zm.ZM_EINVAL
        with pytest.raises(zm.ZmError):
            zm.zm_moments(p.h, [], out)
        assert zm.lib().zm_moments(p.h, None, 1, out.data_ptr(), 0, None) == zm.ZM_EINVAL
        assert zm.lib().zm_reconstruct(p.h, None, 1, out.data_ptr(), 0, None) == zm.ZM_EINVAL


# ------------------------------------------------------------------ full size (4K, bench launch shape)
def test_4k_bench_configuration_sampled():
    # 3840x2160 blob frames, n_max 100, 1024 x 1024 grid, batch 16 as timed by
    # the benchmark; images 0 and 15 are checked in full against the oracle.
    B = 16
    imgs = [synth.blob_image(2160, 3840, 32, workload=2, index=b) for b in (0, 15)]
    others = [torch.rand((2160, 3840), device=DEV) for _ in range(B - 2)]
    with Plan(100, 1024, 1024) as p:
        ts = [dev(imgs[0])] + others + [dev(imgs[1])]
        out = torch.empty((B, p.P, 2), device=DEV)
        zm.zm_moments(p.h, ts, out)
        torch.cuda.synchronize()
        Z = as_complex(out)
        for b, img in ((0, imgs[0]), (B - 1, imgs[1])):
            assert metrics.rel_max_err(Z[b], oracle_moments(img, p)) <= TOL_Z


def test_4k_bench_step_bf16x3_sampled():
    """The step bench.py times, in its launch configuration: zm_moments on 16 4K
    frames with a bf16x3 plan; frames 0 and 15 against the oracle at the split
    form's bar (2e-5 max|Z|).  Then the reconstruction step the bench times
    beside it: zm_moments_ex (polar samples kept) -> zm_reconstruct_errors
    (Neumann), with the reconstruction of the GPU's moments on sampled rings
    against the oracle's Eq. 9, and Eq. 10 / Eq. 13 against sums over the GPU's
    own polar samples and reconstruction."""
    B, n_max, n_rho, n_theta = 16, 100, 1024, 1024
    imgs = [synth.blob_image(2160, 3840, 32, workload=2, index=b) for b in (0, 15)]
    others = [torch.rand((2160, 3840), device=DEV) for _ in range(B - 2)]
    with Plan(n_max, n_rho, n_theta, zm.ZM_PREC_BF16X3) as p:
        ts = [dev(imgs[0])] + others + [dev(imgs[1])]
        fhat = torch.empty((B, n_rho, n_theta), device=DEV)
        out = torch.empty((B, p.P, 2), device=DEV)
        frec = torch.empty((B, n_rho, n_theta), device=DEV)
        err = torch.empty((B, 4), device=DEV, dtype=torch.float64)
        zm.zm_moments(p.h, ts, out, 0)
        torch.cuda.synchronize()
        Zm = as_complex(out)
        for b, img in ((0, imgs[0]), (B - 1, imgs[1])):
            assert metrics.rel_max_err(Zm[b], oracle_moments(img, p)) <= 2e-5, b
        zm.zm_moments_ex(p.h, ts, out, fhat, 0)
        zm.zm_reconstruct_errors(p.h, out, B, frec, fhat, err, zm.ZM_NEUMANN)
        torch.cuda.synchronize()
        Z = as_complex(out)
        assert np.array_equal(Z, Zm)
        e = err.cpu().numpy()
        rings = np.array([0, 1, 7, 8, 255, 512, 1000, 1023])
        rho, _ = grid.radial_nodes(n_rho)
        k = np.arange(n_theta)[None, :]
        m = np.arange(n_max + 1)[:, None]
        basis = np.cos(2 * np.pi * ((m * k) % n_theta) / n_theta) + 1j * np.sin(2 * np.pi * ((m * k) % n_theta) / n_theta)
        for b, img in ((0, imgs[0]), (B - 1, imgs[1])):
            assert metrics.rel_max_err(Z[b], oracle_moments(img, p)) <= TOL_Z, b
            rec_ref = (orc.radial_spectrum(Z[b], n_max, rho[rings], neumann=True) @ basis).real
            got = frec[b, rings].double().cpu().numpy()
            assert np.max(np.abs(got - rec_ref)) <= 1e-4 * np.max(np.abs(rec_ref)), b
            f = fhat[b].double().cpu().numpy()
            r = frec[b].double().cpu().numpy()
            sd = np.sum((f - r) ** 2)
            assert abs(e[b, 0] - sd / np.sum(f * f)) <= 1e-4 * e[b, 0], b
            assert abs(e[b, 1] - sd / (f.max() ** 2 * f.size)) <= 1e-4 * e[b, 1], b
            assert e[b, 3] == n_rho * n_theta


# ------------------------------------------------------------------ host frames -> disk boxes
@pytest.mark.parametrize("pinned", [True, False])
def test_upload_disk_boxes_give_the_same_moments(pinned):
    """zm_upload_disk copies only the disk's row spans (plus the bilinear
    margin) of host frames into their bounding boxes; moments from the boxes
    match moments from the whole frames on the device (float rounding of the
    shifted coordinates only).  The device buffer starts as NaN, so a pixel
    read outside the copied spans would show in the moments."""
    frames = [synth.blob_image(270, 480, 6, workload=70, index=b) for b in range(3)]
    geos = [None, (250.0, 140.0, 100.0), (20.5, 30.0, 60.0)]      # centred, off-centre, clipped by the edge
    host = [torch.from_numpy(f).pin_memory() if pinned else torch.from_numpy(f) for f in frames]
    with Plan(40, 64, 128, zm.ZM_PREC_BF16X3) as p:
        nbytes = zm.zm_upload_disk_bytes(host, geometries=geos)
        assert zm.zm_upload_disk_traffic(host, geometries=geos) < nbytes
        dev_buf = torch.full((nbytes // 4 + 4,), float("nan"), device=DEV)
        try:
            boxes = zm.zm_upload_disk(host, dev_buf, geometries=geos)
        except zm.ZmError as e:                                  # pageable memory on a device that cannot read it
            assert not pinned and e.status == zm.ZM_EUNSUPPORTED
            pytest.skip("pageable host memory is not readable by this device")
        torch.cuda.synchronize()
        assert sum(b.height * b.width for b in boxes) < 3 * 270 * 480
        got = torch.empty((3, p.P, 2), device=DEV)
        zm.zm_moments(p.h, boxes, got)
        want = gpu_moments(p, frames, geometries=geos)
        torch.cuda.synchronize()
        g = as_complex(got)
    for b in range(3):
        assert metrics.rel_max_err(g[b], want[b]) <= 1e-5, b
        ref = om.moments(frames[b].astype(np.float64), 40, 64, 128,
                         geometry=geos[b] if geos[b] else None)
        assert metrics.rel_max_err(g[b], ref) <= TOL_Z, b


# ------------------------------------------------------------------ high orders on Gauss-Legendre nodes
@pytest.mark.parametrize("prec", [zm.ZM_PREC_FP32, zm.ZM_PREC_BF16X3])
@pytest.mark.parametrize("npr,mpr", [(480, 40), (497, 1), (500, 500), (300, 0)])
def test_high_order_polar_closed_form(prec, npr, mpr):
    """Orders up to 500 (the paper's stability range, Sec. 3.1): the polar input
    R_{n'm'}(rho) cos(m' theta) on Gauss-Legendre nodes has the closed-form
    moments 1 (m' = 0) or 1/2 at (n', m') and 0 elsewhere; the table comes from
    Eq. 7, the input from the oracle's Jacobi recurrence."""
    n_max, n_rho, n_theta = 500, 512, 1024
    rho, _ = grid.radial_nodes(n_rho, "gauss")
    th = grid.angles(n_theta)
    R = zernike.zrp(npr, mpr, rho)
    fh = dev((R[:, None] * np.cos(mpr * th)[None, :])[None])
    with Plan(n_max, n_rho, n_theta, prec | zm.ZM_GRID_GAUSS) as p:
        out = torch.empty((1, p.P, 2), device=DEV)
        zm.zm_moments_polar(p.h, fh, 1, out)
        torch.cuda.synchronize()
        Z = as_complex(out)[0]
    want = np.zeros(p.P, complex)
    want[zernike.moment_index(npr, mpr)] = 1.0 if mpr == 0 else 0.5
    assert np.max(np.abs(Z - want)) <= (2e-5 if prec == zm.ZM_PREC_FP32 else 1e-4)


def test_reconstruction_error_does_not_grow_with_order_on_gauss_nodes():
    """With Gauss-Legendre radial nodes (N_rho >= n_max + 1) the discrete
    Zernike functions are orthogonal on the grid, so the reconstruction is a
    projection onto a growing subspace and its error (Eq. 10, Eq. 13 on the
    polar nodes) cannot grow with n_max: no high-order breakdown (Sec. 3.1)."""
    img = synth.blob_image(512, 512, 12, workload=71, index=0)
    n_rho, n_theta = 320, 1024
    eps = []
    for n_max in (20, 60, 120, 200, 300):
        with Plan(n_max, n_rho, n_theta, zm.ZM_PREC_FP32 | zm.ZM_GRID_GAUSS) as p:
            out = torch.empty((1, p.P, 2), device=DEV)
            fh = torch.empty((1, n_rho, n_theta), device=DEV)
            zm.zm_moments_ex(p.h, [dev(img)], out, fh)
            err = torch.empty((1, 4), device=DEV, dtype=torch.float64)
            zm.zm_reconstruct_errors(p.h, out, 1, None, fh, err, zm.ZM_NEUMANN)
            torch.cuda.synchronize()
            eps.append(float(err[0, 0]))
    assert all(b <= a * (1 + 1e-3) for a, b in zip(eps, eps[1:])), eps
    assert eps[-1] < 0.5 * eps[0], eps


# ------------------------------------------------------------------ colour frames (three bands)
def test_colour_frame_as_three_bands_matches_oracle():
    """A colour frame is a batch of its three bands (Sec. 2.3, Sec. 3): per-band
    min / max over the disk kept, moments and the Cartesian reconstruction of
    each band, the reconstruction min-max normalised to its band's stored range
    (Table I), and Eq. 10 / Eq. 13 per band."""
    h, w = 64, 80
    bands = [synth.blob_image(h, w, 4 + c, workload=72, index=c) * (0.5 + 0.25 * c) for c in range(3)]
    n_max, n_rho, n_theta = 20, 32, 64
    mask = metrics.disk_mask(h, w)
    with Plan(n_max, n_rho, n_theta) as p:
        db = [dev(b) for b in bands]
        mm = torch.empty((3, 2), device=DEV)
        zm.zm_disk_minmax(p.h, db, mm)
        out = torch.empty((3, p.P, 2), device=DEV)
        zm.zm_moments(p.h, db, out)
        canv = [torch.zeros((h, w), device=DEV) for _ in range(3)]
        polar = torch.empty((3, n_rho, n_theta), device=DEV)
        zm.zm_reconstruct_cartesian(p.h, out, canv, polar, zm.ZM_NEUMANN)
        zm.zm_minmax_normalize(p.h, canv, mm)
        err = torch.empty((3, 4), device=DEV, dtype=torch.float64)
        zm.zm_errors(p.h, db, canv, err)
        torch.cuda.synchronize()
        Z = as_complex(out)
    rho, _ = grid.radial_nodes(n_rho)
    geo = grid.default_geometry(h, w)
    y, x = np.mgrid[0:h, 0:w]
    r_xy, _ = grid.pixel_to_polar(x, y, geo)
    inner = mask & (np.abs(r_xy - 1.0) > 1e-5)
    for c in range(3):
        f = bands[c].astype(np.float64)
        lo, hi = f[mask].min(), f[mask].max()
        assert abs(float(mm[c, 0]) - lo) <= 1e-6 and abs(float(mm[c, 1]) - hi) <= 1e-6
        Zref = oracle_moments(bands[c], p)
        assert metrics.rel_max_err(Z[c], Zref) <= TOL_Z
        polar_ref = orc.reconstruct_polar(Zref, n_max, n_rho, n_theta, neumann=True)
        ref = metrics.minmax_normalize(orc.polar_to_cartesian(polar_ref, rho, h, w), lo, hi, mask)
        got = canv[c].double().cpu().numpy()
        assert np.max(np.abs(got[inner] - ref[inner])) <= 1e-3 * (hi - lo), c
        e = err[c].cpu().numpy()
        # the errors of the GPU's own normalised band, and against the oracle's
        assert abs(e[0] - metrics.eps1(f, got, mask)) <= 1e-4 * e[0]
        assert abs(e[1] - metrics.eps13(f, got, mask)) <= 1e-4 * e[1]
        assert abs(e[1] - metrics.eps13(f, ref, mask)) <= 5e-2 * e[1]


# ------------------------------------------------------------------ Cartesian summation (Eq. 3-6)
from oracle import cartesian as ocart  # noqa: E402

CART_PAIRS = [(0, 0), (1, 1), (2, 0), (5, 3), (20, 12), (40, 40), (37, 1), (63, 59), (100, 6)]


def cart_gpu(imgs, pairs, geos=None, flags=0):
    ts = [dev(i) for i in imgs]
    out = torch.empty((len(ts), len(pairs), 2), device=DEV)
    work = torch.empty(zm.zm_cartesian_work_bytes(len(ts), len(pairs)) // 8 + 1, dtype=torch.float64, device=DEV)
    zm.zm_cartesian_moments(ts, pairs, out, work, flags, geometries=geos)
    torch.cuda.synchronize()
    return as_complex(out)


def cart_bound(img, geo, n):
    # |R e^{-j m theta}| <= 1: the moment's natural scale, for FP32 rounding
    rows, cols, _, _ = ocart.disk_pixels(*img.shape, geo)
    return (n + 1) / (np.pi * geo[2] ** 2) * np.sum(np.abs(img[rows, cols]))


@pytest.mark.parametrize("h,w,geo", [
    (64, 64, None),                      # half offset: 8-point orbits
    (63, 63, None),                      # integer offset: orbits with v = 0 and u = v
    (60, 75, None),                      # cx integer, cy half: one thread per pixel
    (50, 70, (30.5, 20.5, 18.0)),        # explicit disk inside the image
    (40, 40, (10.5, 12.5, 30.0)),        # disk reaching past the edges (zero outside)
    (45, 52, (20.3, 21.7, 15.5))])       # off-grid centre: per pixel
def test_cartesian_matches_oracle(h, w, geo):
    img = synth.blob_image(h, w, 5, workload=73, index=h + w)
    got = cart_gpu([img], CART_PAIRS, [geo] if geo else None)[0]
    g = geo if geo else grid.default_geometry(h, w)
    ref = ocart.moments_cartesian(img, CART_PAIRS, g)
    for k, (n, m) in enumerate(CART_PAIRS):
        assert abs(got[k] - ref[k]) <= 2e-6 * cart_bound(img.astype(np.float64), g, n), (n, m, got[k], ref[k])


def test_cartesian_batches_pairs_and_neumann():
    imgs = [synth.blob_image(48 + 2 * b, 48 + 2 * b, 4, workload=74, index=b) for b in range(10)]
    pairs = [(4, 0), (7, 3), (12, 8), (9, 1), (30, 0), (2, 2)]
    plain = cart_gpu(imgs, pairs)
    neu = cart_gpu(imgs, pairs, flags=zm.ZM_NEUMANN)
    for b, img in enumerate(imgs):
        ref = ocart.moments_cartesian(img, pairs)
        g = grid.default_geometry(*img.shape)
        for k, (n, m) in enumerate(pairs):
            tol = 2e-6 * cart_bound(img.astype(np.float64), g, n)
            assert abs(plain[b, k] - ref[k]) <= tol
            assert abs(neu[b, k] - ref[k] / (2.0 if m == 0 else 1.0)) <= tol


def test_cartesian_large_frame_single_moment():
    img = synth.blob_image(2048, 2048, 24, workload=75, index=0)
    pairs = [(100, 36), (99, 1)]
    got = cart_gpu([img], pairs)[0]
    ref = ocart.moments_cartesian(img, pairs)
    g = grid.default_geometry(2048, 2048)
    for k, (n, m) in enumerate(pairs):
        assert abs(got[k] - ref[k]) <= 2e-6 * cart_bound(img.astype(np.float64), g, n)


def test_cartesian_argument_errors():
    img = dev(np.ones((16, 16), np.float32))
    out = torch.empty((1, 1, 2), device=DEV)
    work = torch.empty(zm.zm_cartesian_work_bytes(1, 1) // 8 + 1, dtype=torch.float64, device=DEV)
    for bad in ([(3, 2)], [(2, 3)], [(-1, 1)], [(1030, 0)]):
        with pytest.raises(zm.ZmError) as e:
            zm.zm_cartesian_moments([img], bad, out, work)
        assert e.value.status == zm.ZM_EINVAL
    with pytest.raises(zm.ZmError) as e:
        zm.zm_cartesian_moments([img], [(2, 0)], out, work[:2])
    assert e.value.status == zm.ZM_EINVAL


@pytest.mark.parametrize("n_max,n_rho,n_theta", [(20, 32, 64), (100, 96, 1024), (500, 16, 2048), (3, 9, 8)])
def test_ring_spectra_cross_check_against_cufft(n_max, n_rho, n_theta):
    """The warp FFT's ring spectra against the vendor FFT (torch.fft on the
    device, i.e. cuFFT) of the same polar samples: a cross-check only, the
    product path never calls it."""
    img = synth.blob_image(2 * n_rho + 4, 2 * n_rho + 2, 5, workload=76, index=n_theta)
    with Plan(n_max, n_rho, n_theta) as p:
        F = torch.empty((n_max + 1, 1, 2, n_rho), device=DEV)
        fh = torch.empty((1, n_rho, n_theta), device=DEV)
        zm.zm_ring_spectra(p.h, [dev(img)], F, fh)
        ref = torch.fft.rfft(fh[0].double(), dim=-1)[:, : n_max + 1]          # [i][m], e^{-j m theta_k}
        torch.cuda.synchronize()
    got = torch.complex(F[:, 0, 0, :].double(), F[:, 0, 1, :].double()).T     # [i][m]
    err = (got - ref).abs().max().item()
    assert err <= 2e-6 * ref.abs().max().item() * np.log2(n_theta), err


# ------------------------------------------------------------------ the two stages of zm_moments
@pytest.mark.parametrize("prec", [zm.ZM_PREC_FP32, zm.ZM_PREC_BF16X3, zm.ZM_PREC_FP16X3])
def test_stage_calls_equal_zm_moments(prec):
    imgs = [synth.blob_image(256, 320, 8, workload=26, index=b) for b in range(3)]
    ts = [dev(i) for i in imgs]
    with Plan(40, 100, 128, prec) as p:
        a = torch.empty((3, p.P, 2), device=DEV)
        b = torch.empty((3, p.P, 2), device=DEV)
        zm.zm_moments(p.h, ts, a, zm.ZM_NEUMANN)
        zm.zm_stage_spectra(p.h, ts)
        zm.zm_stage_project(p.h, 3, b, zm.ZM_NEUMANN)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        with pytest.raises(zm.ZmError) as e:
            zm.zm_stage_project(p.h, 2, b)
        assert e.value.status == zm.ZM_EINVAL
    ref = oracle_moments(imgs[1], p, neumann=True)
    assert metrics.rel_max_err(as_complex(a)[1], ref) <= TOL_Z
