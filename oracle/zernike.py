"""Zernike index set and radial polynomials (oracle; test infrastructure only).

Sec. 2, Eq. 1-2: a moment Z_nm exists for n >= 0, |m| <= n, n - |m| even, and
Z_{n,-m} = conj(Z_nm), so only m >= 0 is stored.  Eq. 2 defines R_nm by a
factorial sum; Sec. 2.1 (Eq. 7-8) gives the DFT-of-Chebyshev-U identity that
the fast method uses.
"""

from fractions import Fraction
from math import factorial

import numpy as np


def index_pairs(n_max):
    """All stored (n, m) pairs in storage order: n ascending, then m ascending,
    m >= 0 with n - m even (Eq. 1 conditions; negative m follow from
    Z_{n,-m} = conj(Z_nm))."""
    pairs = []
    for n in range(n_max + 1):
        for m in range(n % 2, n + 1, 2):
            pairs.append((n, m))
    return pairs


def num_moments(n_max):
    """Number of stored moments up to order n_max (by enumeration)."""
    return len(index_pairs(n_max))


def moment_index(n, m):
    """Position of (n, m) in the storage order of ``index_pairs``."""
    if m < 0 or m > n or (n - m) % 2:
        raise ValueError("invalid (n, m)")
    return index_pairs(n).index((n, m))


def zrp_exact(n, m, rho):
    """R_nm(rho) by the factorial sum of Eq. 2, in exact rational arithmetic.

    ``rho`` is a Fraction (or int); the result is a Fraction.
    """
    m = abs(m)
    if m > n or (n - m) % 2:
        return Fraction(0)
    rho = Fraction(rho)
    total = Fraction(0)
    for s in range((n - m) // 2 + 1):
        num = factorial(n - s) * (-1) ** s
        den = factorial((n - m) // 2 - s) * factorial((n + m) // 2 - s) * factorial(s)
        total += Fraction(num, den) * rho ** (n - 2 * s)
    return total


def _jacobi_0b(s_max, beta, x):
    """P_s^{(0,beta)}(x) for s = 0..s_max by the three-term recurrence of the
    Jacobi polynomials (DLMF 18.9.1-18.9.2 with alpha = 0).  Returns a list of
    arrays, one per degree."""
    x = np.asarray(x, dtype=np.float64)
    out = [np.ones_like(x)]
    if s_max >= 1:
        out.append(1.0 + (beta + 2.0) * (x - 1.0) / 2.0)
    for s in range(1, s_max):
        a = 2.0 * s + beta
        a1 = 2.0 * (s + 1) * (s + beta + 1) * a
        a2 = -(a + 1.0) * beta * beta
        a3 = a * (a + 1.0) * (a + 2.0)
        a4 = 2.0 * s * (s + beta) * (a + 2.0)
        out.append(((a2 + a3 * x) * out[s] - a4 * out[s - 1]) / a1)
    return out


def zrp(n, m, rho):
    """R_n^m(rho) for one pair, by the same recurrence as zrp_table (the table's
    row for (n, m) without the other rows)."""
    rho = np.asarray(rho, dtype=np.float64)
    return rho ** m * _jacobi_0b((n - m) // 2, float(m), 2.0 * rho * rho - 1.0)[(n - m) // 2]


def zrp_table(n_max, rho):
    """R_nm(rho_i) for every stored (n, m) up to n_max, float64.

    Uses R_n^m(rho) = rho^m P_s^{(0,m)}(2 rho^2 - 1), s = (n - m)/2, with the
    Jacobi polynomial from its stable three-term recurrence.  This is the
    definition of Eq. 2 in a numerically stable form (Eq. 2 itself loses all
    digits in float64 at high order, Sec. 1 and Sec. 2).

    Returns an array [P(n_max), len(rho)] in ``index_pairs`` order.
    """
    rho = np.asarray(rho, dtype=np.float64)
    x = 2.0 * rho * rho - 1.0
    pairs = index_pairs(n_max)
    table = np.zeros((len(pairs), rho.size), dtype=np.float64)
    per_m = {}
    for m in range(n_max + 1):
        s_max = (n_max - m) // 2
        per_m[m] = _jacobi_0b(s_max, float(m), x)
    for row, (n, m) in enumerate(pairs):
        table[row] = rho ** m * per_m[m][(n - m) // 2]
    return table


def chebyshev_u(n_max, x):
    """U_0..U_{n_max} at x by U_{n+1} = 2x U_n - U_{n-1} (exact at x = +-1,
    where the sine-ratio form of Eq. 8 is 0/0)."""
    x = np.asarray(x, dtype=np.float64)
    u = [np.ones_like(x)]
    if n_max >= 1:
        u.append(2.0 * x)
    for n in range(1, n_max):
        u.append(2.0 * x * u[n] - u[n - 1])
    return u


def zrp_eq7(n, m, rho, n_points):
    """R_nm(rho) by the DFT identity of Eq. 7: the mean over k of
    U_n(rho cos(2 pi k/N)) cos(2 pi m k/N), k = 0..N-1, float64.

    Reading of the extracted text: the doubled "cos cos" / "sin sin" are read as
    single cos / sin.  The identity is exact when N > n + |m| (no alias of a
    different repetition folds onto m).  Used only to pin those readings.
    """
    k = np.arange(n_points)
    j = (m * k) % n_points
    x = np.asarray(rho, dtype=np.float64)[..., None] * np.cos(2.0 * np.pi * k / n_points)
    u = chebyshev_u(n, x)[n]
    return (u * np.cos(2.0 * np.pi * j / n_points)).sum(axis=-1) / n_points
