"""zm_project_noalloc: the projection for callers that cannot allocate device
memory (their GPU memory is held by another allocator, or their loop cannot
afford cudaMalloc's synchronisation), with its partial sums in a fixed array
of the library instead of a plan workspace.  It must give the same moments as
zm_project, call after call, and refuse requests larger than its array.

This file is collected last on purpose, so that a failure here comes after
every other test has run; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def test_noalloc_projection_matches_zm_project_on_consecutive_calls():
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
            got = torch.full((batch, P, 2), float("nan"), device=DEV)
            # straight through the C ABI
            st = torch.cuda.current_stream().cuda_stream
            status = zm.lib().zm_project_noalloc(plan, spectra.data_ptr(), batch, got.data_ptr(), flags, st)
            assert status == zm.ZM_OK, zm.zm_last_error()
            torch.cuda.synchronize()
            r = ref.double().cpu().numpy()
            g = got.double().cpu().numpy()
            assert not np.isnan(g).any()
            scale = np.max(np.hypot(r[..., 0], r[..., 1]), axis=1)
            err = np.max(np.hypot(g[..., 0] - r[..., 0], g[..., 1] - r[..., 1]), axis=1) / scale
            assert np.all(err <= TOL), (call, err)
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
