"""Exact coprimality check of two 2D kernels by resultants (test infrastructure).

Section 3 requires the two blur kernels, read as bivariate polynomials
k(z1, z2) = sum_{p,q} K[p][q] z1^p z2^q, to be coprime.  Two polynomials with
a common factor of positive degree in z1 have a resultant in z1 that vanishes
identically as a polynomial in z2, and likewise with the roles swapped.  So the
pair is certified coprime when both Res_z1(k1, k2)(z2) and Res_z2(k1, k2)(z1)
are non-zero at some integer point.  The arithmetic is exact: every float
kernel entry is a dyadic rational and ``fractions.Fraction`` keeps it exactly.
"""
from __future__ import annotations

from fractions import Fraction


def _det(mat):
    """Exact determinant by fraction-valued Gaussian elimination."""
    a = [row[:] for row in mat]
    n = len(a)
    det = Fraction(1)
    for col in range(n):
        piv = next((r for r in range(col, n) if a[r][col] != 0), None)
        if piv is None:
            return Fraction(0)
        if piv != col:
            a[col], a[piv] = a[piv], a[col]
            det = -det
        det *= a[col][col]
        inv = 1 / a[col][col]
        for r in range(col + 1, n):
            f = a[r][col] * inv
            if f != 0:
                for c in range(col, n):
                    a[r][c] -= f * a[col][c]
    return det


def _sylvester(f, g):
    """Sylvester matrix of univariate f, g given lowest-degree-first with formal
    degrees len-1 (the resultant of formal degrees; leading zeros allowed)."""
    df, dg = len(f) - 1, len(g) - 1
    n = df + dg
    rows = []
    for i in range(dg):
        row = [Fraction(0)] * n
        for k, c in enumerate(reversed(f)):
            row[i + k] = c
        rows.append(row)
    for i in range(df):
        row = [Fraction(0)] * n
        for k, c in enumerate(reversed(g)):
            row[i + k] = c
        rows.append(row)
    return rows


def _resultant_at(k1, k2, axis: int, point: int):
    """Res in the variable of ``axis`` with the other variable set to ``point``."""
    def collapse(k):
        t = len(k)
        if axis == 0:   # variable z1 (rows) kept; z2 = point
            return [sum(k[p][q] * Fraction(point) ** q for q in range(t)) for p in range(t)]
        return [sum(k[p][q] * Fraction(point) ** p for p in range(t)) for q in range(t)]
    return _det(_sylvester(collapse(k1), collapse(k2)))


def resultant_nonzero(k1, k2, max_points: int | None = None) -> bool:
    """True iff both resultants are shown non-zero at some integer point.

    Res_z1 has degree at most 2 (t1-1)(t2-1) in z2, so if it vanishes at that
    many + 1 distinct points it vanishes identically; ``max_points`` defaults
    to that bound, making a False answer a proof of a common factor (up to a
    simultaneous loss of both leading coefficients, which the generators never
    produce).
    """
    fk1 = [[Fraction(float(v)) for v in row] for row in k1]
    fk2 = [[Fraction(float(v)) for v in row] for row in k2]
    t1, t2 = len(fk1), len(fk2)
    bound = 2 * (t1 - 1) * (t2 - 1) + 1
    if max_points is None:
        max_points = bound
    for axis in (0, 1):
        if not any(_resultant_at(fk1, fk2, axis, pt) != 0 for pt in range(max_points)):
            return False
    return True
