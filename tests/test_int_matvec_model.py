"""The arithmetic of the panel kernel's integer mat-vec (MOLGW_FLAG_EIG_TC), restated on the
CPU with exact Python integers, and its error bound.

Each 64 x 64 tile T of A22 is put on its own grid, a = m 2^(e_T - 53) with
m = rint(a 2^(53 - e_T)) and max |a| over the tile below 2^(e_T), split m = h 2^27 + l;
x is put on one grid the same way.  A product is
  a x = [h h_x 2^54 + (h l_x + l h_x) 2^27 + l l_x] 2^(e_T + e_x - 106),
of which the kernel keeps H = sum h h_x and M = sum (h l_x + l h_x) over a thread's four
elements of a row, T = H + round(M / 2^27) in units of 2^(e_T + e_x - 52), moved to the common grid
2^(e_g - 56 + e_x - 52) by exact left shifts and summed exactly, one rounding per row.
The tests check the model against exact rational products: every row within
  n 2^-52 max|a_row| max|x| + (rounding of the float64 result),
and that one grid per tile keeps small off-diagonal tiles accurate where one grid per row
block of tiles would not (the reason the kernel uses per-tile grids).
"""
from fractions import Fraction

import numpy as np
import pytest

TB = 64


def frexp_e(v):
    """e with |v| < 2^e (0 for v = 0), as the kernel's grid exponent."""
    return int(np.frexp(v)[1]) if v > 0 else 0


def to_grid(v, e):
    """rint(v 2^(53 - e)) exactly (ties to even), as a Python int."""
    return int(np.rint(np.ldexp(v, 53 - e)))


def split27(m):
    h = (m + (1 << 26)) >> 27
    return h, m - (h << 27)


def model_matvec(A, x, grid="tile"):
    """y = A x with the kernel's integer arithmetic (grid = 'tile' or 'rowblock')."""
    n = A.shape[0]
    nb = -(-n // TB)
    ex = frexp_e(np.abs(x).max())
    xs = [split27(to_grid(v, ex)) for v in x]
    e_tile = np.zeros((nb, nb), dtype=int)
    for R in range(nb):
        for J in range(nb):
            blk = A[R * TB:(R + 1) * TB, J * TB:(J + 1) * TB]
            e_tile[R, J] = frexp_e(np.abs(blk).max())
    if grid == "rowblock":
        for R in range(nb):
            e_tile[R, :] = e_tile[R, :].max()
    eg = int(e_tile.max())
    ref = eg - 56
    y = np.empty(n)
    for r in range(n):
        R = r // TB
        acc = 0
        for J in range(nb):
            e = int(e_tile[R, J])
            s = e - ref
            for c0 in range(J * TB, min(n, (J + 1) * TB), 4):    # a thread's four columns
                H = M = 0
                for c in range(c0, min(n, c0 + 4)):
                    h, l = split27(to_grid(A[r, c], e))
                    hx, lx = xs[c]
                    H += h * hx
                    M += h * lx + l * hx
                T = H + ((M + (1 << 26)) >> 27)
                acc += T << s if s >= 0 else T >> min(-s, 63)
        y[r] = float(Fraction(acc) * Fraction(2) ** (ref - 52 + ex))
    return y


def exact_matvec(A, x):
    return np.array([float(sum(Fraction(a) * Fraction(b) for a, b in zip(row, x))) for row in A])


@pytest.mark.parametrize("n,seed", [(70, 0), (130, 1)])
def test_integer_matvec_within_its_bound(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n))
    A = (X + X.T) / 2
    x = rng.standard_normal(n)
    y = model_matvec(A, x)
    ye = exact_matvec(A, x)
    bound = n * 2.0 ** -52 * np.abs(A).max(axis=1) * np.abs(x).max() + 2.0 ** -52 * np.abs(ye)
    assert np.all(np.abs(y - ye) <= bound)
    # and as accurate as a float64 mat-vec in the normwise sense
    assert np.max(np.abs(y - ye)) <= 4 * np.max(np.abs(A @ x - ye)) + 1e-15 * np.abs(ye).max()


def test_per_tile_grids_keep_small_tiles_accurate():
    """A graded matrix: O(1) diagonal tiles, off-diagonal tiles of 1e-6.  One grid per row
    block puts the small tiles on the grid of the large ones (2^-53 of 1, i.e. ~2^-33 of
    their own size); one grid per tile keeps them to 2^-53 of themselves."""
    n = 128
    rng = np.random.default_rng(5)
    X = rng.standard_normal((n, n)) * 1e-6
    A = (X + X.T) / 2
    for R in range(n // TB):
        B = rng.standard_normal((TB, TB))
        A[R * TB:(R + 1) * TB, R * TB:(R + 1) * TB] = (B + B.T) / 2
    x = np.zeros(n)
    x[TB:] = rng.standard_normal(n - TB)          # only the second column block: rows 0..63
    rows = slice(0, TB)                           # see the off-diagonal tile alone
    ye = exact_matvec(A[rows], x)
    err_tile = np.max(np.abs(model_matvec(A, x, "tile")[rows] - ye))
    err_block = np.max(np.abs(model_matvec(A, x, "rowblock")[rows] - ye))
    scale = np.abs(ye).max()
    assert err_tile <= 1e-15 * scale
    assert err_block > 1e3 * err_tile
