"""The two-stage tridiagonalisation prototype (tests/twostage_proto.py): the band and the
tridiagonal it produces are what they claim to be, and their eigenvalues are the input's."""
import numpy as np
import pytest
import scipy.linalg as sl

import twostage_proto as ts


@pytest.mark.parametrize("n,b,seed", [(40, 4, 0), (100, 8, 1), (130, 16, 2)])
def test_band_then_tridiagonal_keep_the_spectrum(n, b, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n))
    A = (X + X.T) / 2
    nrm = np.abs(np.linalg.eigvalsh(A)).max()
    B = ts.band_reduce(A, b)
    assert np.abs(np.tril(B, -b - 1)).max() <= 1e-14 * nrm          # banded
    assert np.abs(B - B.T).max() <= 1e-13 * nrm                       # still symmetric
    T, count = ts.bulge_chase(B, b)
    assert np.abs(np.tril(T, -2)).max() <= 1e-14 * nrm                # tridiagonal
    assert count == ts.reflector_count(n, b)
    w = sl.eigvalsh_tridiagonal(np.diag(T).copy(), np.diag(T, -1).copy())
    assert np.max(np.abs(np.sort(w) - np.linalg.eigvalsh(A))) <= 1e-13 * nrm
    # a diagonal matrix passes through unchanged
    D = np.diag(np.arange(n, dtype=float))
    assert np.array_equal(ts.bulge_chase(ts.band_reduce(D, b), b)[0], D)


def test_cost_model_at_the_bench_order():
    c = ts.cost_model(6400, 64)
    assert c["stage1_flops"] == pytest.approx(4.0 / 3.0 * 6400 ** 3)
    assert c["stage2_flops"] == pytest.approx(6.0 * 6400 ** 2 * 64)
    assert c["stage2_flops"] < 0.05 * c["stage1_flops"]          # 4.5 %: the flops are in stage 1
    assert c["chase_steps"] == 3 * 6400 + 100
    assert ts.reflector_count(640, 64) == pytest.approx(640 ** 2 / (2 * 64), rel=0.15)
