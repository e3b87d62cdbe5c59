"""GPU parity of the tensor-core projection (bf16 / fp16 hi+lo split, FP32
accumulate) against the FP64 oracle and the FP32 path, through the C ABI.

Stated bound for the split forms: max|Z - Z_oracle| <= 1e-4 max|Z_oracle|
(the same bar as FP32; the split keeps ~16 (bf16) / ~22 (fp16) significant
bits of each operand, so the measured error is far below it).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import metrics, moments as om  # noqa: E402
from paper_2304_14492_gb300 import native as zm, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-4
PRECS = {"bf16x3": zm.ZM_PREC_BF16X3, "fp16x3": zm.ZM_PREC_FP16X3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2304_14492_gb300.build import build
    build()
    zm.lib()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def run(n_max, n_rho, n_theta, flags, imgs, call_flags=0):
    plan = zm.zm_plan(n_max, n_rho, n_theta, flags)
    try:
        P = zm.zm_num_moments(n_max)
        out = torch.empty((len(imgs), P, 2), device=DEV)
        zm.zm_moments(plan, [dev(i) for i in imgs], out, call_flags)
        zm.zm_plan_status(plan)                      # no bounded wait gave up
        o = out.double().cpu().numpy()
        return o[..., 0] + 1j * o[..., 1]
    finally:
        zm.zm_plan_destroy(plan)


@pytest.mark.parametrize("prec", sorted(PRECS))
@pytest.mark.parametrize("n_max,n_rho,n_theta,shape,batch", [
    (20, 32, 64, (64, 64), 1),          # small plan, one column tile
    (50, 256, 256, (512, 512), 16),     # 32 columns
    (13, 37, 32, (45, 70), 70),         # ragged N_rho, 140 columns -> 2 column tiles
    (300, 24, 1024, (48, 48), 3),       # K_0 = 151 -> N = 160 (256 TMEM columns)
    (600, 8, 2048, (16, 16), 2),        # K_0 = 301 -> two order tiles
    (0, 5, 8, (10, 10), 1),             # single moment
])
def test_tensor_projection_matches_oracle(prec, n_max, n_rho, n_theta, shape, batch):
    imgs = [synth.blob_image(shape[0], shape[1], 4, workload=20, index=b) if b % 2 == 0
            else synth.uniform_image(shape[0], shape[1], workload=20, index=b) for b in range(batch)]
    Z = run(n_max, n_rho, n_theta, PRECS[prec], imgs)
    check = range(batch) if batch <= 4 else (0, 1, batch // 2, batch - 1)
    for b in check:
        ref = om.moments(imgs[b].astype(np.float64), n_max, n_rho, n_theta)
        assert metrics.rel_max_err(Z[b], ref) <= TOL, (prec, b)


@pytest.mark.parametrize("prec", sorted(PRECS))
def test_tensor_projection_neumann_and_polar(prec):
    rng = np.random.default_rng(9)
    n_max, n_rho, n_theta = 30, 48, 64
    fh = rng.random((5, n_rho, n_theta)).astype(np.float32) * 200.0     # large grey levels (fp16 scaling)
    plan = zm.zm_plan(n_max, n_rho, n_theta, PRECS[prec])
    try:
        P = zm.zm_num_moments(n_max)
        out = torch.empty((5, P, 2), device=DEV)
        zm.zm_moments_polar(plan, dev(fh), 5, out, zm.ZM_NEUMANN)
        zm.zm_plan_status(plan)
        o = out.double().cpu().numpy()
    finally:
        zm.zm_plan_destroy(plan)
    for b in range(5):
        ref = om.moments_polar(fh[b].astype(np.float64), n_max, neumann=True)
        assert metrics.rel_max_err(o[b, :, 0] + 1j * o[b, :, 1], ref) <= TOL


def test_tensor_vs_fp32_path_4k_frame():
    img = synth.blob_image(2160, 3840, 32, workload=2, index=0)
    z32 = run(100, 1024, 1024, zm.ZM_PREC_FP32, [img])[0]
    ref = om.moments(img.astype(np.float64), 100, 1024, 1024)
    assert metrics.rel_max_err(z32, ref) <= TOL
    for prec in PRECS.values():
        zt = run(100, 1024, 1024, prec, [img])[0]
        assert metrics.rel_max_err(zt, ref) <= TOL
        assert metrics.rel_max_err(zt, z32) <= TOL


@pytest.mark.parametrize("neumann", [False, True])
@pytest.mark.parametrize("n_max,n_rho,n_theta,batch", [
    (20, 32, 64, 1),
    (100, 128, 256, 3),
    (150, 40, 512, 2),        # K_0 = 76: two 64-order chunks
    (13, 37, 32, 130),        # ragged rings, 260 columns -> two column tiles
    (0, 3, 8, 1),
])
def test_tensor_reconstruction_matches_oracle(neumann, n_max, n_rho, n_theta, batch):
    """bf16 plans reconstruct with the tensor-core radial contraction; bar
    1e-4 max|f~| (the hi+lo split keeps ~16 significant bits per operand)."""
    from oracle import reconstruct as orc
    rng = np.random.default_rng(n_max + batch)
    P = zm.zm_num_moments(n_max)
    Z = rng.normal(size=(batch, P)) + 1j * rng.normal(size=(batch, P))
    Z = Z.astype(np.complex64)
    plan = zm.zm_plan(n_max, n_rho, n_theta, zm.ZM_PREC_BF16X3)
    try:
        zin = dev(np.stack([Z.real, Z.imag], -1))
        out = torch.empty((batch, n_rho, n_theta), device=DEV)
        zm.zm_reconstruct(plan, zin, batch, out, zm.ZM_NEUMANN if neumann else 0)
        zm.zm_plan_status(plan)
        got = out.double().cpu().numpy()
    finally:
        zm.zm_plan_destroy(plan)
    for b in (range(batch) if batch <= 4 else (0, 1, 64, 129)):
        ref = orc.reconstruct_polar(Z[b].astype(np.complex128), n_max, n_rho, n_theta, neumann=neumann)
        assert np.max(np.abs(got[b] - ref)) <= 1e-4 * np.max(np.abs(ref)), b
