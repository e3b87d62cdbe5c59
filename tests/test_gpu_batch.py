"""GPU parity of uneven batches (zm_batch_*): images of mixed sizes, orders
and polar grids in one graph launch, against the FP64 oracle, with replay and
re-capture checks and the autotuner's cache file."""

import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import metrics, moments as om  # noqa: E402
from paper_2304_14492_gb300 import native as zm, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2304_14492_gb300.build import build
    build()
    zm.lib()


def make_batch(count, workload=40):
    specs = synth.uneven_batch_specs(count=count, workload=workload)
    imgs, items, outs = [], [], []
    for j, (size, n_max, n_rho, n_theta) in enumerate(specs):
        img = synth.blob_image(size, size, 8, workload=workload, index=j)
        t = torch.from_numpy(img).to(DEV)
        out = torch.full((zm.zm_num_moments(n_max), 2), float("nan"), device=DEV)
        imgs.append(img)
        items.append((t, n_max, n_rho, n_theta, out))
        outs.append(out)
    return specs, imgs, items, outs


@pytest.mark.parametrize("prec", [zm.ZM_PREC_FP32, zm.ZM_PREC_BF16X3, zm.ZM_PREC_FP16X3])
def test_uneven_batch_matches_oracle_and_replays(prec, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("ZM_TUNE_CACHE", str(cache))
    specs, imgs, items, outs = make_batch(24)
    batch = zm.zm_batch_create(items, prec)
    try:
        info = zm.zm_batch_info(batch)
        assert info["groups"] == len({(s[2], s[3]) for s in specs})
        zm.zm_batch_run(batch, items)
        torch.cuda.synchronize()
        first = [o.clone() for o in outs]
        # one sample per (size, N_theta) cell against the oracle
        seen = set()
        for j, (size, n_max, n_rho, n_theta) in enumerate(specs):
            if (size, n_theta) in seen:
                continue
            seen.add((size, n_theta))
            o = outs[j].double().cpu().numpy()
            assert not np.isnan(o).any()
            ref = om.moments(imgs[j].astype(np.float64), n_max, n_rho, n_theta)
            assert metrics.rel_max_err(o[:, 0] + 1j * o[:, 1], ref) <= TOL, (j, size, n_max)
        # replay with the same pointers: no new capture, same results
        for o in outs:
            o.fill_(float("nan"))
        zm.zm_batch_run(batch, items)
        torch.cuda.synchronize()
        assert zm.zm_batch_info(batch)["captures"] == 1
        for a, b in zip(first, outs):
            assert torch.equal(a, b)
        # new output buffers: captured again, same results
        items2 = [(t, n, r, k, torch.empty_like(o)) for (t, n, r, k, o) in items]
        zm.zm_batch_run(batch, items2)
        torch.cuda.synchronize()
        assert zm.zm_batch_info(batch)["captures"] == 2
        for a, it in zip(first, items2):
            assert torch.equal(a, it[4])
        zm.zm_batch_run(batch, items2, zm.ZM_NEUMANN)
        torch.cuda.synchronize()
        for (size, n_max, _, _), a, it in zip(specs, first, items2):
            want = a.clone()
            want[[zm.zm_index(n, 0) for n in range(0, n_max + 1, 2)]] *= 0.5
            assert torch.allclose(it[4], want, rtol=0, atol=0)
    finally:
        zm.zm_batch_destroy(batch)
    entries = json.load(open(cache))
    assert len(entries) == info["groups"]
    for v in entries.values():
        assert v["rings"] in (2, 4, 8) and v["split"] in (4, 8) and v["gather"] in (0, 1)


def test_batch_with_unaligned_image_and_shape_check():
    big = torch.from_numpy(synth.blob_image(140, 140, 6, workload=41, index=0)).to(DEV)
    view = big[3:131, 1:129]                            # unaligned base: fused gather path
    out_a = torch.empty((zm.zm_num_moments(40), 2), device=DEV)
    out_b = torch.empty((zm.zm_num_moments(30), 2), device=DEV)
    aligned = torch.from_numpy(synth.blob_image(128, 128, 6, workload=41, index=1)).to(DEV)
    items = [(view, 40, 64, 128, out_a), (aligned, 30, 64, 128, out_b)]
    batch = zm.zm_batch_create(items, zm.ZM_PREC_FP32)
    try:
        zm.zm_batch_run(batch, items)
        torch.cuda.synchronize()
        for img, (t, n_max, n_rho, n_theta, out) in zip([view, aligned], items):
            ref = om.moments(img.double().cpu().numpy(), n_max, n_rho, n_theta)
            o = out.double().cpu().numpy()
            assert metrics.rel_max_err(o[:, 0] + 1j * o[:, 1], ref) <= TOL
        bad = [(view, 41, 64, 128, out_a), (aligned, 30, 64, 128, out_b)]
        with pytest.raises(zm.ZmError) as e:
            zm.zm_batch_run(batch, bad)
        assert e.value.status == zm.ZM_EINVAL
    finally:
        zm.zm_batch_destroy(batch)
