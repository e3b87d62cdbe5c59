"""zm_project_noalloc: the projection for callers that cannot allocate device
memory (their GPU memory is held by another allocator, or their loop cannot
afford cudaMalloc's synchronisation), with its partial sums in a fixed array
of the library instead of a plan workspace.  It must give the same moments as
zm_project and as the oracle's radial projection of the same spectra, call
after call, compute in FP32 whatever the plan's precision, stay right when the
array forces a single radial slice, and refuse requests larger than its array.

This file is collected last on purpose, so that a failure here comes after
every other test has run; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grid, moments as om  # noqa: E402
from paper_2304_14492_gb300 import native as zm, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-4          # the moment tolerance used by the parity tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2304_14492_gb300.build import build
    build()
    zm.lib()


def noalloc(plan, spectra, batch, P, flags):
    """One call straight through the C ABI."""
    got = torch.full((batch, P, 2), float("nan"), device=DEV)
    st = torch.cuda.current_stream().cuda_stream
    status = zm.lib().zm_project_noalloc(plan, spectra.data_ptr(), batch, got.data_ptr(), flags, st)
    assert status == zm.ZM_OK, zm.zm_last_error()
    return got


def rel_err(got, ref):
    """max |got - ref| / max |ref| per image."""
    g, r = got.double().cpu().numpy(), ref.double().cpu().numpy()
    assert not np.isnan(g).any()
    scale = np.max(np.hypot(r[..., 0], r[..., 1]), axis=1)
    return np.max(np.hypot(g[..., 0] - r[..., 0], g[..., 1] - r[..., 1]), axis=1) / scale


def oracle_projection(spectra, b, n_max, n_rho, n_theta, neumann):
    """The oracle's Eq. 1 quadrature of image b's spectra (copied to the host)."""
    s = spectra.double().cpu().numpy()
    F = (s[:, b, 0, :] + 1j * s[:, b, 1, :]).T            # [N_rho, n_max + 1]
    rho, wr = grid.radial_nodes(n_rho)
    Z = om.project(F, wr, n_theta, n_max, rho=rho, neumann=neumann)
    return np.stack([Z.real, Z.imag], axis=-1)[None]


def test_noalloc_projection_matches_zm_project_and_oracle_on_consecutive_calls():
    n_max, n_rho, n_theta = 50, 256, 256
    plan = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_FP32)
    try:
        P = zm.zm_num_moments(n_max)
        for call, (batch, flags) in enumerate([(4, 0), (7, zm.ZM_NEUMANN)]):
            imgs = [torch.from_numpy(synth.blob_image(512, 512, 8, workload=30, index=10 * call + b)).to(DEV)
                    for b in range(batch)]
            spectra = torch.empty((n_max + 1, batch, 2, n_rho), device=DEV)
            zm.zm_ring_spectra(plan, imgs, spectra)
            ref = torch.empty((batch, P, 2), device=DEV)
            zm.zm_project(plan, spectra, batch, ref, flags)
            got = noalloc(plan, spectra, batch, P, flags)
            torch.cuda.synchronize()
            assert np.all(rel_err(got, ref) <= TOL), call
            for b in (0, batch - 1):
                o = torch.from_numpy(oracle_projection(spectra, b, n_max, n_rho, n_theta, bool(flags)))
                assert rel_err(got[b:b + 1], o)[0] <= TOL, (call, b)
    finally:
        zm.zm_plan_destroy(plan)


def test_noalloc_projection_on_a_bf16_plan_computes_in_fp32():
    """A bf16x3 plan's call gives the FP32 plan's zm_project moments to FP32
    rounding (both run the FP32 split-K kernels on the same FP32 table)."""
    n_max, n_rho, n_theta = 40, 128, 256
    P = zm.zm_num_moments(n_max)
    p32 = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_FP32)
    p16 = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_BF16X3)
    try:
        batch = 3
        imgs = [torch.from_numpy(synth.blob_image(256, 256, 8, workload=31, index=b)).to(DEV) for b in range(batch)]
        spectra = torch.empty((n_max + 1, batch, 2, n_rho), device=DEV)
        zm.zm_ring_spectra(p32, imgs, spectra)
        ref = torch.empty((batch, P, 2), device=DEV)
        zm.zm_project(p32, spectra, batch, ref, 0)
        got = noalloc(p16, spectra, batch, P, 0)
        torch.cuda.synchronize()
        assert np.all(rel_err(got, ref) <= 1e-6)
    finally:
        zm.zm_plan_destroy(p16)
        zm.zm_plan_destroy(p32)


def test_noalloc_projection_near_its_limit_uses_one_slice():
    """P(200) * 2 * 64 = 1,305,728 floats: one radial slice fits the array, two
    do not, so the whole radial sum runs in one slice."""
    n_max, n_rho, n_theta, batch = 200, 64, 512, 64
    P = zm.zm_num_moments(n_max)
    assert P * 2 * batch <= 1 << 21 < 2 * P * 2 * batch
    plan = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_FP32)
    try:
        imgs = [torch.from_numpy(synth.blob_image(128, 128, 4, workload=32, index=b)).to(DEV) for b in range(batch)]
        spectra = torch.empty((n_max + 1, batch, 2, n_rho), device=DEV)
        zm.zm_ring_spectra(plan, imgs, spectra)
        ref = torch.empty((batch, P, 2), device=DEV)
        zm.zm_project(plan, spectra, batch, ref, 0)
        for _ in range(2):
            got = noalloc(plan, spectra, batch, P, 0)
            torch.cuda.synchronize()
            assert np.all(rel_err(got, ref) <= TOL)
        o = torch.from_numpy(oracle_projection(spectra, batch - 1, n_max, n_rho, n_theta, False))
        assert rel_err(got[batch - 1:], o)[0] <= TOL
    finally:
        zm.zm_plan_destroy(plan)


def test_noalloc_projection_rejects_requests_beyond_its_array():
    n_max, n_rho, n_theta = 200, 8, 512          # P = 10201 moments
    plan = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_FP32)
    try:
        batch = 128                               # 10201 * 256 floats > 2^21
        spectra = torch.zeros((n_max + 1, batch, 2, n_rho), device=DEV)
        out = torch.empty((batch, zm.zm_num_moments(n_max), 2), device=DEV)
        with pytest.raises(zm.ZmError) as e:
            zm.zm_project_noalloc(plan, spectra, batch, out)
        assert e.value.status == zm.ZM_EINVAL
        assert "fixed scratch" in str(e.value)
    finally:
        zm.zm_plan_destroy(plan)
