"""GPU tests of the serving loop (zm_server_*): continuous batching of host
requests under an HBM budget.  Each result must be the same alone and in the
mix (within the moment tolerance), requests that arrive while others run must
be admitted and overlap, and the oracle must agree on a sample."""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import metrics, moments as om  # noqa: E402
from paper_2304_14492_gb300 import native as zm, synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2304_14492_gb300.build import build
    build()
    zm.lib()
    torch.cuda.init()


def next_pow2(x):
    p = 1
    while p < x:
        p *= 2
    return p


def make_requests(count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for j in range(count):
        size = int(rng.choice([64, 128, 256, 512]))
        n_max = int(rng.choice([20, 50, 100]))
        img = synth.blob_image(size, size, 6, workload=50 + seed, index=j)
        reqs.append((img, n_max, size // 2, next_pow2(2 * n_max + 2)))
    return reqs


def run_server(reqs, budget, streams=4, max_group=16, prec=zm.ZM_PREC_FP32, alone=False, max_wait_us=0):
    srv = zm.zm_server_create(budget, streams, max_group, prec, max_wait_us)
    outs = [np.full((zm.zm_num_moments(n), 2), np.nan, np.float32) for (_, n, _, _) in reqs]
    try:
        if alone:
            for (img, n, r, k), o in zip(reqs, outs):
                t = zm.zm_server_submit(srv, img, n, r, k, o)
                zm.zm_server_wait(srv, t, 30.0)
        else:
            tickets = [zm.zm_server_submit(srv, img, n, r, k, o) for (img, n, r, k), o in zip(reqs, outs)]
            zm.zm_server_drain(srv, 60.0)
            assert all(zm.zm_server_poll(srv, t) for t in tickets)
        stats = zm.zm_server_stats(srv)
    finally:
        zm.zm_server_destroy(srv, 30.0)
    return outs, stats


@pytest.mark.parametrize("prec", [zm.ZM_PREC_FP32, zm.ZM_PREC_BF16X3])
def test_alone_equals_mix_and_oracle(prec):
    reqs = make_requests(40, seed=1)
    alone, st_a = run_server(reqs, 256 << 20, prec=prec, alone=True)
    # a 20 ms batching window: the 40 submissions (12 grids) form groups
    mix, st_m = run_server(reqs, 256 << 20, prec=prec, max_wait_us=20000)
    assert st_a["completed"] == st_m["completed"] == len(reqs)
    assert st_a["groups_launched"] == len(reqs)
    assert st_m["groups_launched"] < len(reqs)                   # requests were batched
    for (img, n, r, k), a, m in zip(reqs, alone, mix):
        za = a[:, 0] + 1j * a[:, 1]
        zm_ = m[:, 0] + 1j * m[:, 1]
        assert not np.isnan(za).any() and not np.isnan(zm_).any()
        assert metrics.rel_max_err(zm_, za) <= 1e-5
    for j in (0, 7, 21, 39):
        img, n, r, k = reqs[j]
        ref = om.moments(img.astype(np.float64), n, r, k)
        zz = mix[j][:, 0] + 1j * mix[j][:, 1]
        assert metrics.rel_max_err(zz, ref) <= TOL
    assert st_m["p99_ms"] >= st_m["p50_ms"] > 0


def test_tight_budget_admits_as_memory_frees_and_stays_correct():
    reqs = make_requests(30, seed=2)
    big = max(img.nbytes for img, *_ in reqs)
    budget = 3 * big                                            # only a few requests fit at once
    outs, st = run_server(reqs, budget, max_group=4, max_wait_us=2000)
    ref, _ = run_server(reqs, 256 << 20)
    assert st["completed"] == len(reqs)
    assert st["peak_bytes"] <= budget
    for a, b in zip(outs, ref):
        assert metrics.rel_max_err(a[:, 0] + 1j * a[:, 1], b[:, 0] + 1j * b[:, 1]) <= 1e-5


def test_arrivals_while_busy_and_errors():
    srv = zm.zm_server_create(64 << 20, 2, 8, zm.ZM_PREC_FP32)
    try:
        img = synth.blob_image(256, 256, 6, workload=60, index=0)
        outs = []
        tickets = []
        t0 = time.perf_counter()
        for j in range(50):                                     # a steady trickle of arrivals
            o = np.zeros((zm.zm_num_moments(50), 2), np.float32)
            outs.append(o)
            tickets.append(zm.zm_server_submit(srv, img, 50, 128, 128, o))
            time.sleep(0.0005)
        zm.zm_server_drain(srv, 30.0)
        assert time.perf_counter() - t0 < 30
        z0 = outs[0][:, 0] + 1j * outs[0][:, 1]
        for o in outs[1:]:                                      # groups of any size: same moments
            assert metrics.rel_max_err(o[:, 0] + 1j * o[:, 1], z0) <= 1e-5
        too_big = np.zeros((8192, 8192), np.float32)            # 256 MiB > budget
        with pytest.raises(zm.ZmError) as e:
            zm.zm_server_submit(srv, too_big, 10, 64, 32, np.zeros((zm.zm_num_moments(10), 2), np.float32))
        assert e.value.status == zm.ZM_ENOMEM
        with pytest.raises(zm.ZmError) as e:
            zm.zm_server_submit(srv, img, 50, 128, 64, np.zeros((zm.zm_num_moments(50), 2), np.float32))
        assert e.value.status == zm.ZM_EINVAL                  # n_theta < 2 n_max + 1
        st = zm.zm_server_stats(srv)
        assert st["completed"] == 50 and st["rejected"] == 1
    finally:
        zm.zm_server_destroy(srv, 30.0)


def test_mixed_arrivals_every_size_order_cell_matches_oracle():
    """Requests drawn from the serving mix (sizes 256/512/1024 and a 2160x2160
    centred crop of a 3840x2160 frame; n_max 20/50/100/200; N_rho = size/2,
    N_theta = next power of two >= 2 n_max + 2) arrive while earlier ones run;
    one request of every (size, n_max) cell is checked against the oracle, and
    every request against the same request served alone."""
    rng = np.random.default_rng(11)
    frame = synth.blob_image(2160, 3840, 32, workload=61, index=0)
    pool = {2160: np.ascontiguousarray(frame[:, 840:3000])}
    for sz in (256, 512, 1024):
        pool[sz] = synth.blob_image(sz, sz, 8, workload=61, index=sz)
    cells = [(sz, n) for sz in (256, 512, 1024, 2160) for n in (20, 50, 100, 200)]
    order = cells + [cells[int(k)] for k in rng.integers(0, len(cells), 48)]
    reqs = [(pool[sz], n, sz // 2, next_pow2(2 * n + 2)) for sz, n in order]
    srv = zm.zm_server_create(2 << 30, 4, 32, zm.ZM_PREC_BF16X3)
    outs = [np.full((zm.zm_num_moments(n), 2), np.nan, np.float32) for (_, n, _, _) in reqs]
    try:
        for (img, n, r, k), o in zip(reqs, outs):
            zm.zm_server_submit(srv, img, n, r, k, o)
            time.sleep(float(rng.exponential(0.0005)))
        zm.zm_server_drain(srv, 120.0)
        st = zm.zm_server_stats(srv)
    finally:
        zm.zm_server_destroy(srv, 60.0)
    assert st["completed"] == len(reqs)
    alone, _ = run_server(reqs, 2 << 30, prec=zm.ZM_PREC_BF16X3, alone=True)
    for a, m in zip(alone, outs):
        assert metrics.rel_max_err(m[:, 0] + 1j * m[:, 1], a[:, 0] + 1j * a[:, 1]) <= 1e-5
    for j, (sz, n) in enumerate(cells):
        img, n, r, k = reqs[j]
        ref = om.moments(img.astype(np.float64), n, r, k)
        assert metrics.rel_max_err(outs[j][:, 0] + 1j * outs[j][:, 1], ref) <= TOL, (sz, n)


def test_reset_stats_only_when_drained():
    srv = zm.zm_server_create(64 << 20, 1, 4, zm.ZM_PREC_FP32, 50000)
    try:
        img = synth.blob_image(128, 128, 4, workload=62, index=0)
        o = np.zeros((zm.zm_num_moments(20), 2), np.float32)
        zm.zm_server_submit(srv, img, 20, 64, 64, o)       # held by the 50 ms window
        with pytest.raises(zm.ZmError) as e:
            zm.zm_server_reset_stats(srv)
        assert e.value.status == zm.ZM_EINVAL
        zm.zm_server_drain(srv, 10.0)
        assert zm.zm_server_stats(srv)["completed"] == 1
        zm.zm_server_reset_stats(srv)
        st = zm.zm_server_stats(srv)
        assert st["completed"] == 0 and st["submitted"] == 0 and st["p99_ms"] == 0
    finally:
        zm.zm_server_destroy(srv, 10.0)


def test_direct_host_access_and_pinned_staging_agree(monkeypatch):
    """The two copy paths (kernels on the callers' host buffers where the GPU
    reaches pageable host memory, else a pinned mirror) give identical results."""
    reqs = make_requests(12, seed=5)
    direct, st_d = run_server(reqs, 256 << 20)
    monkeypatch.setenv("ZM_SERVER_STAGING", "1")
    staged, st_s = run_server(reqs, 256 << 20)
    assert st_s["host_direct"] == 0
    for a, b in zip(direct, staged):
        assert metrics.rel_max_err(a[:, 0] + 1j * a[:, 1], b[:, 0] + 1j * b[:, 1]) <= 1e-5
