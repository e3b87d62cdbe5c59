"""The C-ABI library builds, loads and exports every entry point the header
declares; host-only helpers agree with the oracle's index set (CPU)."""

import ctypes
import os
import re

import pytest

from oracle import zernike

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "zm.h")


@pytest.fixture(scope="module")
def zm():
    from paper_2304_14492_gb300 import build as b
    from paper_2304_14492_gb300 import native
    b.build()
    native.lib()
    return native


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9 \*]*?\b(zm_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("zm_plan", "zm_moments", "zm_reconstruct", "zm_plan_destroy", "zm_strerror",
                     "zm_num_moments", "zm_index", "zm_moments_polar"):
        assert required in names


def test_library_exports_every_declared_symbol(zm):
    L = ctypes.CDLL(zm.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in zm.SIGNATURES, name
    assert set(zm.SIGNATURES) == set(declared_functions())


def test_index_helpers_match_oracle(zm):
    for n_max in range(0, 60):
        assert zm.zm_num_moments(n_max) == zernike.num_moments(n_max)
    for row, (n, m) in enumerate(zernike.index_pairs(40)):
        assert zm.zm_index(n, m) == row
    assert zm.zm_index(3, 2) == -1 and zm.zm_index(2, 4) == -1 and zm.zm_index(-1, 0) == -1
    assert zm.zm_num_moments(-1) == -1
    assert zm.zm_strerror(0) == "ok" and zm.zm_strerror(1) == "invalid argument"


def test_plan_argument_errors_are_reported_not_raised(zm):
    # argument validation happens before any device call
    for args in [(-1, 8, 8), (4, 0, 16), (4, 8, 12), (10, 8, 16), (4, 8, 4096)]:
        with pytest.raises(zm.ZmError) as e:
            zm.zm_plan(*args)
        assert e.value.status in (zm.ZM_EINVAL, zm.ZM_EUNSUPPORTED)
    with pytest.raises(zm.ZmError):
        zm.zm_plan(4, 8, 16, 0x2)          # unknown grid flag


def test_no_gpu_plan_fails_cleanly(zm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(zm.ZmError) as e:
        zm.zm_plan(4, 8, 16)
    assert e.value.status == zm.ZM_ECUDA


@pytest.mark.parametrize("geo", [None, (150.5, 100.0, 80.0), (30.0, 40.5, 70.0)])
def test_upload_traffic_lies_between_the_stencils_and_the_box(zm, geo):
    """zm_upload_disk_traffic (host logic, no GPU): at least the bytes of the
    columns the bilinear stencils of the oracle's polar samples touch in each
    row (from the 4-aligned first column), at most that plus the spans' margins,
    and less than the bounding box; centred, off-centre and edge-clipped disks."""
    import numpy as np
    from oracle import grid
    h, w, n_rho, n_theta = 270, 480, 135, 512
    img = np.zeros((h, w), np.float32)
    host = [img]
    geos = [geo] if geo else None
    traffic = zm.zm_upload_disk_traffic(host, geometries=geos)
    box = zm.zm_upload_disk_bytes(host, geometries=geos)
    rho, _ = grid.radial_nodes(n_rho)
    theta = 2 * np.pi * np.arange(n_theta) / n_theta
    X, Y = grid.polar_to_pixel(rho[:, None], theta[None, :], geo if geo else grid.default_geometry(h, w))
    x0, y0 = np.floor(X).astype(int).ravel(), np.floor(Y).astype(int).ravel()
    lo, hi = {}, {}
    for dy in (0, 1):
        for dx in (0, 1):
            xs, ys = x0 + dx, y0 + dy
            ok = (xs >= 0) & (xs < w) & (ys >= 0) & (ys < h)
            for x, y in zip(xs[ok], ys[ok]):
                lo[y] = min(lo.get(y, x), x)
                hi[y] = max(hi.get(y, x), x)
    need = sum(4 * (hi[y] - (lo[y] & ~3) + 1) for y in lo)
    assert need <= traffic <= need + 4 * 12 * len(lo) + 4 * 12 * 4
    assert traffic < box
