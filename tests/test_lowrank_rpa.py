"""The low-rank (secular) route to the RPA poles, prototyped in lowrank_rpa.py, gives
the oracle's Omega and residue weights on small workloads; its cost model says why
the library keeps the dense reduction (no GPU needed)."""
import numpy as np
import pytest

import lowrank_rpa as lr
import synthetic as sy
from oracle import qsgw


@pytest.mark.parametrize("nb,no,na,seed", [(24, 5, 72, 0), (12, 3, 40, 5)])
def test_secular_route_matches_the_oracle(nb, no, na, seed):
    m = sy.molecule(nb, no, na, seed)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, sy.ETA)
    D, V = lr.low_rank_factors(r["B"], m["eps"], no)
    np.testing.assert_allclose(D, r["D"], rtol=0, atol=0)
    np.testing.assert_allclose(D[:, None] ** 2 * np.eye(len(D)) + V @ V.T, r["M"], rtol=1e-12,
                               atol=1e-13 * np.abs(r["M"]).max())
    lam = lr.secular_eigvals(D * D, V)
    np.testing.assert_allclose(np.sqrt(lam), r["Omega"], rtol=1e-12)
    R = lr.secular_residue_weights(lam, D, V)
    np.testing.assert_allclose(R, r["R"], rtol=1e-7, atol=1e-9 * np.abs(r["R"]).max())


def test_count_is_the_inertia_of_the_formed_matrix():
    rng = np.random.default_rng(4)
    n, k = 40, 6
    D2 = np.sort(rng.uniform(0.2, 9.0, n))
    V = rng.standard_normal((n, k))
    ev = np.linalg.eigvalsh(np.diag(D2) + V @ V.T)
    for lam in np.linspace(0.1, ev.max() + 1.0, 37):
        assert lr.count_below(lam, D2, V) == int(np.sum(ev < lam))


@pytest.mark.parametrize("nb", [200, 400, 600])
def test_cost_model_at_the_workloads(nb):
    """With n_occ = nb/5 and n_aux = 3 nb both routes scale as nb^6: the secular route
    stays ~10^3 times the dense one at every size of this shape."""
    no, na = nb // 5, 3 * nb
    c = lr.cost_model(no * (nb - no), na)
    assert 5e2 < c["ratio"] < 5e3
