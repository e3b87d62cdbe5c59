"""The error bound of the split-precision projection, checked in CPU arithmetic.

The tensor-core projection of Eq. 1 computes each product a*f of a weight
a = (n+1)/pi * w_i * 2pi/N_theta * R_nm(rho_i) and a spectrum value f as
a_hi f_hi + a_hi f_lo + a_lo f_hi, where x_hi is x rounded to the 16-bit format
(p significant bits: 8 for bf16, 11 for fp16) and x_lo is x - x_hi rounded
again.  With u = 2^-p:

    |x - x_hi - x_lo| <= u^2 |x|,      |x_lo| <= u |x|,

so one product is off by at most |a_lo f_lo| + |a_hi||f - f_hi - f_lo| +
|a - a_hi - a_lo||f_hi| <= 3 u^2 |a f| (to first order), and the moment

    |Z_split - Z| <= 3 u^2 S_nm,   S_nm = sum_i |a_i| |f_i|

(3 * 2^-16 * 2^-2 = 3 * 2^-18 for bf16, 3 * 2^-22 for fp16), before the FP32
rounding of the accumulation.  The products here are emulated exactly (float64
holds every product of two 16-bit values and their short sums), so the test
sees the split alone: the bf16 and fp16 splits stay inside the bound on the
64x64 and 512x512 workloads, and splits that keep less (a shorter lo part, a
dropped cross term, no lo part) break it, so the bound detects them.  The
stacked form of the projection, which also forms a_lo f_lo, has the tighter
bound (2 u^2 + u^4) S_nm, checked the same way.
"""

import numpy as np
import pytest

from paper_2304_14492_gb300 import synth
from splitmath import dft_matrix, dft_split_spectra, rne, split_moments, terms


WORKLOADS = {
    "64x64 uniform, n_max 20": (lambda: synth.uniform_image(64, 64, workload=0, index=0), (20, 32, 64)),
    "512x512 blobs, n_max 50": (lambda: synth.blob_image(512, 512, 8, workload=1, index=0), (50, 256, 256)),
}


@pytest.fixture(scope="module", params=sorted(WORKLOADS))
def workload(request):
    make, args = WORKLOADS[request.param]
    return terms(make(), *args)


def test_rounding_helper_matches_known_values():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7 at 8 bits: to even -> 1
    assert rne(np.array([1.0 + 2.0 ** -8]), 8)[0] == 1.0
    assert rne(np.array([1.0 + 3 * 2.0 ** -8]), 8)[0] == 1.0 + 2.0 ** -6
    assert rne(np.array([np.pi]), 11)[0] == np.float64(np.float16(np.pi))
    x = np.linspace(-3, 3, 1001)
    assert np.array_equal(rne(x, 11), x.astype(np.float16).astype(np.float64))


@pytest.mark.parametrize("p", [8, 11])
def test_split_stays_inside_its_bound(workload, p):
    a, f, z, S = workload
    err = np.abs(split_moments(a, f, p) - z)
    bound = 3 * 2.0 ** (-2 * p - 2) * S
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("weaker", [dict(lo_bits=4), dict(terms_kept=("hh", "hl")), dict(terms_kept=("hh",))])
def test_weaker_bf16_splits_break_the_bound(workload, weaker):
    a, f, z, S = workload
    err = np.abs(split_moments(a, f, 8, **weaker) - z)
    assert np.max(err / (3 * 2.0 ** -18 * S)) > 1.0


# When every order has at most 64 rows the blocked projection stacks A hi and
# A lo on the MMA's M and multiplies both by [F hi | F lo], so it also forms
# a_lo f_lo.  With e_a = a - a_hi - a_lo and e_f = f - f_hi - f_lo,
#     a f - (a_hi + a_lo)(f_hi + f_lo) = a e_f + e_a f - e_a e_f,
# so the four products are off by at most (2 u^2 + u^4) |a f| per term, a
# bound inside the three-product one (the errors themselves need not shrink
# term by term: rounding errors of the three-product form can cancel).
@pytest.mark.parametrize("p", [8, 11])
def test_four_product_split_stays_inside_its_tighter_bound(workload, p):
    a, f, z, S = workload
    u2 = 2.0 ** (-2 * p)
    err4 = np.abs(split_moments(a, f, p, terms_kept=("hh", "hl", "lh", "ll")) - z)
    assert np.all(err4 <= (2 * u2 + u2 * u2) * S), float(np.max(err4 / ((2 * u2 + u2 * u2) * S)))
    assert np.all(err4 <= 3 * u2 * S)


# ---- the angular sums as a split product (the tensor-core DFT kernel)
#
# F_m(rho_i) = sum_k f_ik w_mk with |w_mk| = 1; the split drops at most
# 3 u^2 |f_ik| per term (same argument as above, per real component, and the
# two components together stay inside it by the triangle inequality), so
#
#     |F_split - F| <= 3 u^2 sum_k |f_ik|.

DFT_WORKLOADS = {
    "64x64 uniform, N_theta 64": (lambda: synth.uniform_image(64, 64, workload=0, index=0), (20, 32, 64)),
    "512x512 blobs, N_theta 256": (lambda: synth.blob_image(512, 512, 8, workload=1, index=0), (50, 256, 256)),
}


@pytest.fixture(scope="module", params=sorted(DFT_WORKLOADS))
def dft_workload(request):
    from oracle import grid, moments as om, resample
    make, (n_max, n_rho, n_theta) = DFT_WORKLOADS[request.param]
    img = make().astype(np.float64)
    rho, _ = grid.radial_nodes(n_rho)
    fh = resample.polar_resample(img, rho, n_theta, grid.default_geometry(*img.shape))
    return fh, n_max, om.angular_dft(fh, n_max), np.sum(np.abs(fh), axis=1)[:, None]


def test_dft_matrix_is_the_oracles_angular_transform(dft_workload):
    fh, n_max, F, _ = dft_workload
    c, s = dft_matrix(n_max, fh.shape[1])
    assert np.allclose(fh @ c.T + 1j * (fh @ s.T), F, rtol=0, atol=1e-12 * np.max(np.abs(F)))


@pytest.mark.parametrize("p", [8, 11])
def test_dft_split_stays_inside_its_bound(dft_workload, p):
    fh, n_max, F, L1 = dft_workload
    err = np.abs(dft_split_spectra(fh, n_max, p) - F)
    assert np.all(err <= 3 * 2.0 ** (-2 * p) * L1), float(np.max(err / (3 * 2.0 ** (-2 * p) * L1)))


# The bound adds every term's worst case; the rounding errors of the N_theta
# terms have mixed signs, so the real split sits at a few percent of it, and
# of the weaker splits only a lo part of 2 bits or a dropped cross term
# exceeds it (the GPU test of the kernel compares it with this emulation to
# FP32 rounding, which catches the rest).
@pytest.mark.parametrize("weaker", [dict(lo_bits=2), dict(terms_kept=("hh", "hl")), dict(terms_kept=("hh",))])
def test_weaker_dft_splits_break_the_bound(dft_workload, weaker):
    fh, n_max, F, L1 = dft_workload
    err = np.abs(dft_split_spectra(fh, n_max, 8, **weaker) - F)
    assert np.max(err / (3 * 2.0 ** -16 * L1)) > 1.0
