"""Pins of the oracle's index set and radial polynomials (CPU).

Eq. 2 (factorial sum) is checked against hand-expanded closed forms; the
float64 recurrence against Eq. 2 in exact rationals, against scipy's Jacobi
and Legendre routines and against orthogonality on Gauss-Legendre nodes; the
Eq. 7 identity against Eq. 2 (pinning the readings of its garbled text).
"""

from fractions import Fraction

import numpy as np
import pytest
import scipy.special as sp

from oracle import grid, zernike


def test_index_set_counts_and_closed_form():
    # P(n_max) = (q+1)^2 for n_max = 2q and (q+1)(q+2) for n_max = 2q+1.
    for n_max in range(0, 41):
        q = n_max // 2
        want = (q + 1) ** 2 if n_max % 2 == 0 else (q + 1) * (q + 2)
        assert zernike.num_moments(n_max) == want
    assert [zernike.num_moments(n) for n in (20, 50, 80, 100, 200)] == [121, 676, 1681, 2601, 10201]
    # Position of (n, m): off(n) + (m - n mod 2)/2 with off(2q) = q(q+1),
    # off(2q+1) = (q+1)^2.
    for row, (n, m) in enumerate(zernike.index_pairs(30)):
        q = n // 2
        off = q * (q + 1) if n % 2 == 0 else (q + 1) ** 2
        assert row == off + (m - n % 2) // 2
        assert zernike.moment_index(n, m) == row
    with pytest.raises(ValueError):
        zernike.moment_index(3, 2)


# Hand-expanded Eq. 2 for n <= 6: coefficient lists, highest power first,
# of the powers rho^n, rho^(n-2), ...
CLOSED = {
    (0, 0): [1], (1, 1): [1], (2, 0): [2, -1], (2, 2): [1],
    (3, 1): [3, -2], (3, 3): [1], (4, 0): [6, -6, 1], (4, 2): [4, -3],
    (4, 4): [1], (5, 1): [10, -12, 3], (5, 3): [5, -4], (5, 5): [1],
    (6, 0): [20, -30, 12, -1], (6, 2): [15, -20, 6], (6, 4): [6, -5], (6, 6): [1],
}


def closed_form(n, m, rho):
    return sum(c * rho ** (n - 2 * j) for j, c in enumerate(CLOSED[(n, m)]))


@pytest.mark.parametrize("rho", [Fraction(0), Fraction(1, 3), Fraction(5, 7), Fraction(1)])
def test_eq2_exact_matches_hand_expansion(rho):
    for (n, m) in CLOSED:
        assert zernike.zrp_exact(n, m, rho) == closed_form(n, m, rho)
        assert zernike.zrp_exact(n, -m, rho) == closed_form(n, m, rho)


def test_eq2_special_values():
    for n in range(0, 25):
        for m in range(n % 2, n + 1, 2):
            assert zernike.zrp_exact(n, m, 1) == 1                       # R_nm(1) = 1
            if m > 0:
                assert zernike.zrp_exact(n, m, 0) == 0                   # R_nm(0) = 0, m > 0
        assert zernike.zrp_exact(n, n, Fraction(2, 3)) == Fraction(2, 3) ** n   # R_nn = rho^n
        if n % 2 == 0:
            assert zernike.zrp_exact(n, 0, 0) == (-1) ** (n // 2)
        if n >= 1:
            assert zernike.zrp_exact(n, (n + 1) % 2, Fraction(1, 2)) == 0    # n - m odd: no such R


def test_recurrence_vs_exact_all_low_orders():
    # Exhaustive at n <= 12 on the midpoint nodes of N_rho = 16 and on a few
    # other rationals, every (n, m).
    n_rho = 16
    rhos = [Fraction(2 * i + 1, 2 * n_rho) for i in range(n_rho)] + [Fraction(0), Fraction(1), Fraction(3, 11)]
    table = zernike.zrp_table(12, np.array([float(r) for r in rhos]))
    for row, (n, m) in enumerate(zernike.index_pairs(12)):
        for j, r in enumerate(rhos):
            assert abs(table[row, j] - float(zernike.zrp_exact(n, m, r))) <= 1e-14


@pytest.mark.parametrize("n,m", [(100, 0), (100, 36), (101, 1), (200, 10), (200, 150), (500, 10), (500, 300)])
def test_recurrence_vs_exact_high_order(n, m):
    rhos = [Fraction(255, 256), Fraction(1, 2), Fraction(63, 64), Fraction(1, 1024), Fraction(701, 1024)]
    table = zernike.zrp_table(n, np.array([float(r) for r in rhos]))
    row = zernike.index_pairs(n).index((n, m))
    for j, r in enumerate(rhos):
        exact = zernike.zrp_exact(n, m, r)
        # compare against the exact value at the float64 node actually used
        exact_at_node = zernike.zrp_exact(n, m, Fraction(float(r)))
        assert exact == exact_at_node  # dyadic rationals are exact in float64
        assert abs(table[row, j] - float(exact)) <= 1e-13


@pytest.mark.parametrize("n,m", [(0, 0), (7, 3), (100, 36), (500, 10), (500, 500), (499, 1)])
def test_single_pair_vs_exact(n, m):
    # zrp(n, m, .) against the exact rational Eq. 2 at dyadic nodes
    rhos = [Fraction(255, 256), Fraction(1, 2), Fraction(1, 1024), Fraction(701, 1024), Fraction(1)]
    got = zernike.zrp(n, m, np.array([float(r) for r in rhos]))
    for j, r in enumerate(rhos):
        assert abs(got[j] - float(zernike.zrp_exact(n, m, r))) <= 1e-13


def test_recurrence_vs_scipy_jacobi_and_legendre():
    rho = np.linspace(0.0, 1.0, 57)
    n_max = 40
    table = zernike.zrp_table(n_max, rho)
    for row, (n, m) in enumerate(zernike.index_pairs(n_max)):
        s = (n - m) // 2
        # R_n^m(rho) = (-1)^s rho^m P_s^{(m,0)}(1 - 2 rho^2)
        ref = (-1) ** s * rho ** m * sp.eval_jacobi(s, m, 0, 1.0 - 2.0 * rho ** 2)
        assert np.max(np.abs(table[row] - ref)) <= 1e-11
        if m == 0:
            assert np.max(np.abs(table[row] - sp.eval_legendre(s, 2 * rho ** 2 - 1))) <= 1e-12


def test_orthogonality_gauss_legendre_to_order_200():
    # Gram of the sampled ZRPs on Gauss-Legendre nodes: within 1e-10 of
    # diag 1/(2(n+1)) for every m, n <= 200.
    n_max = 200
    rho, wr = grid.radial_nodes(n_max + 2, "gauss")
    table = zernike.zrp_table(n_max, rho)
    pairs = zernike.index_pairs(n_max)
    worst = 0.0
    for m in range(n_max + 1):
        rows = [r for r, (n, mm) in enumerate(pairs) if mm == m]
        ns = np.array([pairs[r][0] for r in rows])
        A = table[rows]
        G = (A * wr) @ A.T
        worst = max(worst, np.max(np.abs(G - np.diag(1.0 / (2.0 * (ns + 1))))))
    assert worst <= 1e-10, worst


def test_midpoint_gram_deviation_is_reported_not_exact():
    # On the midpoint rule the Gram matrix is only approximately diagonal; the
    # deviation shrinks with N_rho (second-order rule).
    devs = []
    for n_rho in (64, 256):
        rho, wr = grid.radial_nodes(n_rho, "midpoint")
        table = zernike.zrp_table(20, rho)
        pairs = zernike.index_pairs(20)
        d = 0.0
        for m in range(21):
            rows = [r for r, (n, mm) in enumerate(pairs) if mm == m]
            ns = np.array([pairs[r][0] for r in rows])
            G = (table[rows] * wr) @ table[rows].T
            d = max(d, np.max(np.abs(G - np.diag(1.0 / (2.0 * (ns + 1))))))
        devs.append(d)
    assert devs[1] < devs[0] / 8


def test_eq7_identity_reading():
    # Eq. 7 read with single cos: exact when N > n + |m|, for all parities.
    for n in range(0, 31):
        npts = 1
        while npts < 2 * n + 2:
            npts *= 2
        for m in range(0, n + 1):
            for r in (Fraction(1, 3), Fraction(7, 8), Fraction(1)):
                v = zernike.zrp_eq7(n, m, float(r), npts)
                want = float(zernike.zrp_exact(n, m, r)) if (n - m) % 2 == 0 else 0.0
                assert abs(v - want) <= 1e-13, (n, m, r)
    # The minimum length 2n+1 also works (N > n + m for all m <= n).
    assert abs(zernike.zrp_eq7(20, 20, 0.75, 41) - 0.75 ** 20) <= 1e-14
    # With N <= n + m an alias folds in and the identity fails.
    assert abs(zernike.zrp_eq7(10, 8, 0.9, 18) - float(zernike.zrp_exact(10, 8, Fraction(9, 10)))) > 1e-3
