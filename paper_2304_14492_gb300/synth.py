"""Seeded synthetic images shaped like the paper's workloads.

The paper measures on one 256x256 RGB photograph (Sec. 3) and times image sizes
up to 4000x4000 (Fig. 5); neither the photograph nor any dataset is used here.
Stand-ins:

* ``uniform_image``: grey levels uniform in [0, 1).
* ``blob_image``: a sum of anisotropic Gaussian blobs whose centres are
  area-uniform in the inscribed disk (radius R sqrt(u), angle 2 pi v), with
  standard deviations uniform in [5, 40] px, orientation uniform in [0, pi),
  amplitude uniform in [0.2, 1], plus Gaussian noise of standard deviation 0.01.

Every image is float32 and comes from numpy's default_rng seeded with
SeedSequence([230414492, workload, index]).  This module holds no part of the
moment arithmetic; both the CUDA path and the CPU oracle take its arrays.
"""

import numpy as np

SEED_BASE = 230414492


def rng_for(workload, index):
    return np.random.default_rng(np.random.SeedSequence([SEED_BASE, int(workload), int(index)]))


def uniform_image(height, width, workload=0, index=0):
    rng = rng_for(workload, index)
    return rng.random((height, width), dtype=np.float32)


def blob_image(height, width, n_blobs, workload=0, index=0, noise=0.01,
               disk=None):
    """Blob image; ``disk`` = (cx, cy, R) of the disk the centres are drawn in
    (default: inscribed and centred)."""
    rng = rng_for(workload, index)
    if disk is None:
        disk = ((width - 1) / 2.0, (height - 1) / 2.0, min(height, width) / 2.0)
    cx, cy, R = disk
    img = np.zeros((height, width), dtype=np.float64)
    for _ in range(n_blobs):
        rr = R * np.sqrt(rng.random())
        ph = 2.0 * np.pi * rng.random()
        bx = cx + rr * np.cos(ph)
        by = cy - rr * np.sin(ph)
        s1, s2 = rng.uniform(5.0, 40.0, size=2)
        ang = rng.uniform(0.0, np.pi)
        amp = rng.uniform(0.2, 1.0)
        ext = 5.0 * max(s1, s2)
        x0 = max(int(np.floor(bx - ext)), 0)
        x1 = min(int(np.ceil(bx + ext)) + 1, width)
        y0 = max(int(np.floor(by - ext)), 0)
        y1 = min(int(np.ceil(by + ext)) + 1, height)
        if x0 >= x1 or y0 >= y1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1]
        dx = xx - bx
        dy = yy - by
        c, s = np.cos(ang), np.sin(ang)
        u = c * dx + s * dy
        v = -s * dx + c * dy
        img[y0:y1, x0:x1] += amp * np.exp(-0.5 * ((u / s1) ** 2 + (v / s2) ** 2))
    img += rng.normal(0.0, noise, size=img.shape)
    return img.astype(np.float32)


def next_pow2(x):
    p = 1
    while p < x:
        p *= 2
    return p


def uneven_batch_specs(count=256, workload=3, sizes=(128, 256, 512, 1024),
                       n_min=30, n_max=80):
    """Per-image (size, n_max, N_rho, N_theta) of the uneven-batch workload:
    size uniform over ``sizes``, n_max uniform in [n_min, n_max],
    N_rho = size / 2, N_theta = next power of 2 >= 2 n_max + 2."""
    rng = rng_for(workload, 10**6)
    specs = []
    for _ in range(count):
        size = int(sizes[rng.integers(len(sizes))])
        n = int(rng.integers(n_min, n_max + 1))
        specs.append((size, n, size // 2, next_pow2(2 * n + 2)))
    return specs
