"""A stalled pipeline ends in a status, not a hang: the bounded mbarrier wait
shared by the tensor-core kernels gives up after its limit, reports
ZM_ETIMEOUT, and the context keeps working."""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_14492_gb300 import native as zm, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2304_14492_gb300.build import build
    build()
    zm.lib()


def test_bounded_wait_times_out_and_the_context_survives():
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda:0")
    t0 = time.perf_counter()
    zm.zm_probe_bounded_wait(status)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert int(status.item()) == zm.ZM_ETIMEOUT
    assert 1.5 < dt < 30.0                                   # the 2 s limit, then a normal return
    img = torch.from_numpy(synth.blob_image(64, 64, 3, workload=80, index=0)).to("cuda:0")
    plan = zm.zm_plan(10, 16, 32, zm.ZM_PREC_BF16X3)
    try:
        out = torch.empty((1, zm.zm_num_moments(10), 2), device="cuda:0")
        zm.zm_moments(plan, [img], out)
        zm.zm_plan_status(plan)
        torch.cuda.synchronize()
        assert np.isfinite(out.cpu().numpy()).all()
    finally:
        zm.zm_plan_destroy(plan)


@pytest.mark.parametrize("prec", [zm.ZM_PREC_FP32, zm.ZM_PREC_BF16X3])
def test_outputs_stay_inside_their_buffers(prec):
    """Every output is written inside its buffer: canary words around the
    moment, polar, reconstruction, error and disk-box buffers stay intact
    (ragged sizes: 3 images, N_rho = 37, an odd n_max)."""
    pad = 64
    canary = 1234.5

    def padded(n, dtype=torch.float32):
        t = torch.full((n + 2 * pad,), canary, dtype=dtype, device="cuda:0")
        return t, t[pad:pad + n]

    def intact(t, n):
        c = t.double().cpu().numpy()
        return np.all(c[:pad] == canary) and np.all(c[pad + n:] == canary)

    n_max, n_rho, n_theta, B = 23, 37, 64, 3
    P = zm.zm_num_moments(n_max)
    frames = [synth.blob_image(90, 70 + 10 * b, 4, workload=81, index=b) for b in range(B)]
    imgs = [torch.from_numpy(f).to("cuda:0") for f in frames]
    plan = zm.zm_plan(n_max, n_rho, n_theta, prec)
    try:
        mo_t, mo = padded(B * P * 2)
        fh_t, fh = padded(B * n_rho * n_theta)
        rc_t, rc = padded(B * n_rho * n_theta)
        er_t, er = padded(B * 4, torch.float64)
        zm.zm_moments_ex(plan, imgs, mo.view(B, P, 2), fh.view(B, n_rho, n_theta))
        zm.zm_resample(plan, imgs, fh.view(B, n_rho, n_theta))
        zm.zm_reconstruct(plan, mo.view(B, P, 2), B, rc.view(B, n_rho, n_theta), zm.ZM_NEUMANN)
        zm.zm_reconstruct_errors(plan, mo.view(B, P, 2), B, rc.view(B, n_rho, n_theta), fh.view(B, n_rho, n_theta),
                                 er.view(B, 4), zm.ZM_NEUMANN)
        host = [torch.from_numpy(f).pin_memory() for f in frames]
        nb = zm.zm_upload_disk_bytes(host)
        bx_t, bx = padded(nb // 4)
        zm.zm_upload_disk(host, bx)
        zm.zm_plan_status(plan)
        torch.cuda.synchronize()
    finally:
        zm.zm_plan_destroy(plan)
    assert intact(mo_t, B * P * 2) and intact(fh_t, B * n_rho * n_theta) and intact(rc_t, B * n_rho * n_theta)
    assert intact(er_t, B * 4) and intact(bx_t, nb // 4)
