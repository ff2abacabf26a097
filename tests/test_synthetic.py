"""The seeded input recipe (``synthetic.py``): draw order, ranges, structure and the
statistics the recipe states, so that both sides of every parity test see the
workload the design describes."""
import numpy as np
import pytest

import synthetic as sy


def test_draw_order_and_reproducibility():
    nb, no, na, seed = 12, 3, 7, 5
    m = sy.molecule(nb, no, na, seed)
    rng = np.random.default_rng(seed)
    eo = np.sort(rng.uniform(-20.0, -0.3, no))
    ev = np.sort(rng.uniform(0.05, 5.0, nb - no))
    q, r = np.linalg.qr(rng.standard_normal((nb, nb)))
    g0 = rng.standard_normal((nb, nb))
    assert np.array_equal(m["eps"], np.concatenate([eo, ev]))
    assert np.array_equal(m["C"], q * np.sign(np.diag(r))[None, :])
    assert np.array_equal(m["L"][0], sy.SIGMA0 * (g0 + g0.T) / np.sqrt(2.0))
    m2 = sy.molecule(nb, no, na, seed)
    assert all(np.array_equal(m[k], m2[k]) for k in ("eps", "C", "L"))


def test_ranges_orthogonality_symmetry():
    m = sy.molecule(30, 6, 20, 9)
    eps, C, L = m["eps"], m["C"], m["L"]
    assert np.all(np.diff(eps[:6]) >= 0) and np.all(np.diff(eps[6:]) >= 0)
    assert -20.0 <= eps[:6].min() and eps[:6].max() <= -0.3
    assert 0.05 <= eps[6:].min() and eps[6:].max() <= 5.0
    np.testing.assert_allclose(C.T @ C, np.eye(30), atol=1e-13)
    assert np.array_equal(L, L.transpose(0, 2, 1))


def test_aux_statistics():
    """Off-diagonal (P|mu nu) ~ N(0, s_P^2) with s_P = 0.5 exp(-P/24); successive
    functions correlate as rho = 0.5 (P = 1) and rho sqrt(1 - rho^2) (P >= 2)."""
    nb, na = 160, 6
    m = sy.molecule(nb, 30, na, 3)
    iu = np.triu_indices(nb, 1)
    X = m["L"][:, iu[0], iu[1]]                     # [na, nb(nb-1)/2] samples
    s = sy.aux_sigma(na)
    n = X.shape[1]
    np.testing.assert_allclose(X.std(axis=1), s, rtol=5.0 / np.sqrt(n))
    Z = X / s[:, None]
    corr = np.mean(Z[1:] * Z[:-1], axis=1)
    want = np.r_[sy.RHO, np.full(na - 2, sy.RHO * np.sqrt(1 - sy.RHO ** 2))]
    np.testing.assert_allclose(corr, want, atol=5.0 / np.sqrt(n))
    assert sy.aux_sigma(25)[24] == pytest.approx(0.5 * np.exp(-1.0), rel=1e-15)


def test_coulomb_gram_is_psd():
    """(mu nu|la ta) = sum_P (P|mu nu)(P|la ta) is a Gram matrix."""
    m = sy.molecule(8, 2, 5, 4)
    V = m["L"].reshape(5, -1)
    ev = np.linalg.eigvalsh(V.T @ V)
    assert ev.min() > -1e-12 * ev.max()


def test_batch_sizes():
    ms = sy.config_molecules("D", seeds=range(100, 116))
    for m in ms:
        nb = m["n_basis"]
        assert 40 <= nb <= 160
        assert m["n_occ"] == int(round(nb / 5)) and m["n_aux"] == 3 * nb
        assert nb == int(np.random.default_rng(m["seed"]).integers(40, 161))
    assert len({m["n_basis"] for m in ms}) > 8      # ragged


def test_named_configs_and_errors():
    a = sy.config_molecules("A")[0]
    assert (a["n_basis"], a["n_occ"], a["n_aux"], a["seed"]) == (24, 5, 72, 0)
    assert sy.CONFIGS["B"][:3] == (200, 40, 600)
    for bad in ((10, 0, 5), (10, 10, 5), (10, 3, 0)):
        with pytest.raises(ValueError):
            sy.molecule(*bad, 0)
    m = sy.molecule(6, 2, 3, 1)
    assert np.array_equal(sy.scale_ri(m, 0.5)["L"], 0.5 * m["L"])
