"""The arithmetic behind opts.row_difference, checked on the host against exact rational
determinants: for G = [A; b] whose last row nearly repeats a shared row a_s (b = a_s + a
perturbation of relative size 1e-13, the near-twin labels of the forced workloads), the
row-difference form det G = (b - a_s) . y, y the cofactors of the last row, is accurate to
a few units in the last place, while an fp64 LU of G loses about log10(kappa) digits."""
from fractions import Fraction

import numpy as np

from oracle_pins import exact_det, rand_c


def _cofactors_last_row(A):
    """y_q = (-1)^(n-1+q) det(A without column q), A (n-1) x n, in fp64 (A well conditioned)."""
    m, n = A.shape
    return np.array([(-1) ** (m + q) * np.linalg.det(np.delete(A, q, axis=1)) for q in range(n)])


def _rel_err(x, ex):
    exc = complex(float(ex[0]), float(ex[1]))
    err = abs(Fraction(x.real) - ex[0]) + abs(Fraction(x.imag) - ex[1])
    return float(err) / abs(exc)


def test_row_difference_is_accurate_where_lu_is_not():
    rng = np.random.default_rng(2111)
    for n in (6, 12, 18):
        for _ in range(3):
            A = rand_c(rng, (n - 1, n))
            s = int(rng.integers(0, n - 1))
            b = A[s] + 1e-13 * rand_c(rng, n)
            G = np.vstack([A, b[None, :]])
            ex = exact_det(G)
            y = _cofactors_last_row(A)
            # the row operation leaves the determinant unchanged; the rounded difference is
            # b - a_s to one rounding per entry
            d_rowdiff = np.dot(b - A[s], y)
            d_lu = np.linalg.det(G)
            e_rd, e_lu = _rel_err(d_rowdiff, ex), _rel_err(d_lu, ex)
            assert e_rd < 1e-10, (n, e_rd)
            assert e_rd < 1e-3 * e_lu, (n, e_rd, e_lu)


def test_row_difference_equals_lemma_without_cancellation():
    """Away from near-singularity the two forms agree to rounding: (b - a_r) . y = b . y for any
    shared row a_r, because a_r . y = 0 (a row of A against the cofactors of [A; b]'s last row
    is the determinant of a matrix with a repeated row)."""
    rng = np.random.default_rng(2112)
    n = 9
    A = rand_c(rng, (n - 1, n))
    b = rand_c(rng, n)
    y = _cofactors_last_row(A)
    G = np.vstack([A, b[None, :]])
    ex = exact_det(G)
    for r in range(n - 1):
        assert _rel_err(np.dot(b - A[r], y), ex) < 1e-12
    assert _rel_err(np.dot(b, y), ex) < 1e-12
