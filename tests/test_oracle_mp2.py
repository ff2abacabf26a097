"""Pins of the qsMP2 part of the oracle (Eqs. Sigma.c.MP2, Sigma.c.qsMP2.real).

The matrix form in ``oracle.qsgw`` (``mp2_factors``, ``sigma_mp2_at``,
``sigma_mp2_rows``, ``qsmp2_pass``) is checked against a closed form worked out by
hand for two levels, against the antisymmetrised second-order expansion over
explicit spin orbitals (``oracle.brute.sigma2_spin_orbital``), against the
printed equation where reading R11 leaves it unchanged, and against invariances.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle import brute, qsgw

ETA = 1e-3


def g_re(x, eta=ETA):
    return x / (x * x + eta * eta)


# --------------------------------------------------------------------------
# Two levels (nb = 2, no = 1, na = 1): one spin-up and one spin-down electron
# in orbital 0.  Only opposite-spin pairs exist, so the second-order exchange
# cancels half of the direct term and
#   Sigma_mn(w) = b^2 [b_m0 b_n0 g(w - e0 + d) + b_m1 b_n1 g(w - e1 - d)],
# d = e1 - e0, b = (01|P), b_mn = (mn|P) for the single aux function.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("vals", [(-0.7, 0.4, 0.3, -0.2, 0.25), (-3.0, 1.5, 0.1, 0.6, 0.9)])
def test_two_level_closed_form(vals):
    e0, e1, b00, b11, b = vals
    L = np.array([[[b00, b], [b, b11]]])
    eps = np.array([e0, e1])
    B = qsgw.ri_mo_transform(L, np.eye(2))
    bm = B[0]
    d = e1 - e0
    for w in (-1.3, 0.2, 2.7):
        want = b * b * (np.outer(bm[:, 0], bm[:, 0]) * g_re(w - e0 + d)
                        + np.outer(bm[:, 1], bm[:, 1]) * g_re(w - e1 - d))
        got = qsgw.sigma_mp2_at(B, eps, 1, ETA, w)
        assert np.allclose(got, want, rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------
# The antisymmetrised second-order expansion over spin orbitals
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed,nb,no,na", [(3, 6, 2, 5), (4, 5, 1, 4), (5, 6, 3, 7)])
def test_spin_orbital_expansion(seed, nb, no, na):
    m = sy.molecule(nb, no, na, seed)
    B = qsgw.ri_mo_transform(m["L"], m["C"])
    g = brute.eri_mo(m["L"], m["C"])
    for w in (m["eps"][0], m["eps"][no], 0.37):
        want = brute.sigma2_spin_orbital(g, m["eps"], no, ETA, w)
        got = qsgw.sigma_mp2_at(B, m["eps"], no, ETA, w)
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_printed_equation_where_reading_r11_keeps_it():
    """Empty p (2p1h): the printed factors are the expansion's.  Occupied p (2h1p):
    the printed exchange factor (pi|an) differs from the expansion's (pa|in),
    which is why reading R11 is needed."""
    m = sy.molecule(6, 2, 5, 8)
    g = brute.eri_mo(m["L"], m["C"])
    w = 0.21
    for part in ("2p1h", "2h1p"):
        printed = brute.sigma_mp2_printed(g, m["eps"], 2, ETA, w, part)
        expansion = brute.sigma2_spin_orbital(g, m["eps"], 2, ETA, w, part)
        rel = np.max(np.abs(printed - expansion)) / np.max(np.abs(expansion))
        if part == "2p1h":
            assert rel <= 1e-12
        else:
            assert rel > 1e-3


# --------------------------------------------------------------------------
# Direct term = MP2 limit of GW; rows; symmetry; scaling; fixed point
# --------------------------------------------------------------------------
def test_direct_term_matches_brute_force():
    m = sy.molecule(6, 2, 5, 9)
    B = qsgw.ri_mo_transform(m["L"], m["C"])
    g = brute.eri_mo(m["L"], m["C"])
    w = -0.4
    nb, no = 6, 2
    i, a = qsgw.transitions(nb, no)
    D = m["eps"][a] - m["eps"][i]
    direct = np.zeros((nb, nb))
    for p in range(nb):
        Ap, _ = qsgw.mp2_factors(B, no, p)
        x = w - m["eps"][p] + (D if p < no else -D)
        direct += 2.0 * (Ap * g_re(x)) @ Ap.T
    want = brute.sigma_mp2_direct(g, m["eps"], no, ETA, w)
    assert np.max(np.abs(direct - want)) <= 1e-12 * np.max(np.abs(want))


def test_rows_are_sigma_at_each_row_energy():
    m = sy.molecule(7, 2, 6, 10)
    B = qsgw.ri_mo_transform(m["L"], m["C"])
    S = qsgw.sigma_mp2_rows(B, m["eps"], 2, ETA)
    for r in range(7):
        row = qsgw.sigma_mp2_at(B, m["eps"], 2, ETA, m["eps"][r])[r]
        assert np.allclose(S[r], row, rtol=1e-13, atol=1e-16)


def test_sigma_symmetric_at_fixed_frequency():
    m = sy.molecule(8, 3, 9, 12)
    B = qsgw.ri_mo_transform(m["L"], m["C"])
    for w in (-2.0, 0.05, 1.1):
        S = qsgw.sigma_mp2_at(B, m["eps"], 3, ETA, w)
        assert np.max(np.abs(S - S.T)) <= 1e-12 * np.max(np.abs(S))


def test_fourth_power_scaling_and_ao_rotation():
    """Sigma^MP2 is second order in v: L -> lam L scales it by lam^4 exactly; an
    orthogonal AO rotation leaves it unchanged in the MO basis."""
    m = sy.molecule(7, 2, 6, 13)
    B = qsgw.ri_mo_transform(m["L"], m["C"])
    S = qsgw.sigma_mp2_rows(B, m["eps"], 2, ETA)
    lam = 0.3
    S2 = qsgw.sigma_mp2_rows(lam * B, m["eps"], 2, ETA)
    assert np.allclose(S2, lam ** 4 * S, rtol=1e-12, atol=0)
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((7, 7)))
    Lr = np.einsum("mi,Pmn,nj->Pij", U, m["L"], U)
    Br = qsgw.ri_mo_transform(Lr, U.T @ m["C"])
    Sr = qsgw.sigma_mp2_rows(Br, m["eps"], 2, ETA)
    assert np.max(np.abs(Sr - S)) <= 1e-12 * np.max(np.abs(S))


def test_qsmp2_fixed_point_without_correlation_strength():
    """With L -> lam L the correlation self-energy falls as lam^4 while J and Sigma_x
    fall as lam^2; in the limit the qsMP2 step returns the HF input (reading R5)."""
    m = sy.molecule(8, 3, 8, 14)
    lam = 1e-4
    r = qsgw.qsmp2_pass(lam * m["L"], m["eps"], m["C"], 3, ETA)
    assert np.max(np.abs(r["eps_new"] - m["eps"])) <= 1e-12
    assert np.max(np.abs(r["sigma_c"] - r["sigma_c"].T)) == 0.0


def test_qsmp2_iterations_keep_orthonormal_orbitals():
    m = sy.molecule(10, 3, 12, 15)
    out = qsgw.qsmp2_iterations(m["L"], m["eps"], m["C"], 3, ETA, 2)
    for r in out:
        C = r["C_new"]
        assert np.allclose(C.T @ C, np.eye(10), atol=1e-12)
        assert np.all(np.diff(r["eps_new"]) >= 0)


def test_golden_regression():
    """The oracle still reproduces the stored small-workload values (tests/golden)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "qsmp2_g0w0_nb24_no5_na72_seed0.json")
    doc = json.load(open(path))
    w = doc["workload"]
    m = sy.molecule(w["n_basis"], w["n_occ"], w["n_aux"], w["seed"])
    r = qsgw.qsmp2_pass(m["L"], m["eps"], m["C"], w["n_occ"], w["eta"])
    np.testing.assert_allclose(r["sigma_c"], doc["qsmp2_sigma_c"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["eps_new"], doc["qsmp2_eps_new"], rtol=1e-12, atol=1e-12)
