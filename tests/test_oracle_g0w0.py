"""Pins of the G0W0 part of the oracle (the diagonal of Eq. Sigma.c.GW, reading R12)."""
import math

import numpy as np
import pytest

import synthetic as sy
from oracle import brute, qsgw

ETA = 1e-3


def g_re(x, eta=ETA):
    return x / (x * x + eta * eta)


def dg_re(x, eta=ETA):
    return (eta * eta - x * x) / (x * x + eta * eta) ** 2


@pytest.mark.parametrize("vals", [(-0.7, 0.4, 0.3, -0.2, 0.25), (-3.0, 1.5, 0.1, 0.6, 0.9)])
def test_two_level_closed_form(vals):
    """nb = 2, no = 1, na = 1: Omega = sqrt(d^2 + 4 d b^2), w_pq = B_pq b sqrt(2 d / Omega)."""
    e0, e1, b00, b11, b = vals
    L = np.array([[[b00, b], [b, b11]]])
    eps = np.array([e0, e1])
    r = qsgw.g0w0_pass(L, eps, np.eye(2), 1, ETA)
    d = e1 - e0
    Om = math.sqrt(d * d + 4.0 * d * b * b)
    xpy = math.sqrt(2.0 * d / Om)
    w = np.array([[b00, b], [b, b11]]) * b * xpy
    sig = np.array([w[p, 0] ** 2 * g_re(eps[p] - e0 + Om) + w[p, 1] ** 2 * g_re(eps[p] - e1 - Om)
                    for p in range(2)])
    dsig = np.array([w[p, 0] ** 2 * dg_re(eps[p] - e0 + Om) + w[p, 1] ** 2 * dg_re(eps[p] - e1 - Om)
                     for p in range(2)])
    np.testing.assert_allclose(r["sigma_c_diag"], sig, rtol=1e-12)
    np.testing.assert_allclose(r["dsigma_c_diag"], dsig, rtol=1e-12)
    # input read as HF: Sigma_x,pp - v_pp = 0 and eps_QP = eps + Z Sigma_c,pp(eps_p)
    np.testing.assert_allclose(r["eps_qp"], eps + sig / (1.0 - dsig), rtol=1e-13)


@pytest.mark.parametrize("seed,nb,no,na", [(21, 6, 2, 5), (22, 9, 3, 12)])
def test_diagonal_matches_brute_force_loops(seed, nb, no, na):
    m = sy.molecule(nb, no, na, seed)
    r = qsgw.g0w0_pass(m["L"], m["eps"], m["C"], no, ETA)
    S = brute.sigma_c_loops(r["w"], m["eps"], r["Omega"], no, ETA)   # row p at eps_p
    np.testing.assert_allclose(r["sigma_c_diag"], np.diag(S), rtol=1e-12, atol=1e-15)


def test_derivative_is_the_slope_of_sigma():
    m = sy.molecule(8, 2, 10, 23)
    r = qsgw.g0w0_pass(m["L"], m["eps"], m["C"], 2, ETA)
    h = 1e-6
    for p in range(8):
        hi = qsgw.sigma_c_at(r["w"], m["eps"], r["Omega"], 2, ETA, m["eps"][p] + h)[p, p]
        lo = qsgw.sigma_c_at(r["w"], m["eps"], r["Omega"], 2, ETA, m["eps"][p] - h)[p, p]
        fd = (hi - lo) / (2 * h)
        assert abs(fd - r["dsigma_c_diag"][p]) <= 1e-5 * max(1.0, abs(fd))


def test_hf_start_and_explicit_h_agree():
    m = sy.molecule(10, 3, 12, 24)
    r = qsgw.g0w0_pass(m["L"], m["eps"], m["C"], 3, ETA)
    assert np.max(np.abs(r["sigma_x_diag"] - r["v_diag"])) < 1e-12
    B = qsgw.ri_mo_transform(m["L"], m["C"])
    r2 = qsgw.g0w0_pass(m["L"], m["eps"], m["C"], 3, ETA, h_mo=qsgw.hf_core_mo(B, m["eps"], 3))
    np.testing.assert_allclose(r2["eps_qp"], r["eps_qp"], rtol=1e-13, atol=1e-13)


def test_linearised_energy_solves_the_qp_equation_to_second_order():
    """The residual of w = eps_p + Sigma_c,pp(w) at the linearised w is second order in
    the shift dw: with L -> lam L the shift scales as lam^4 and Sigma'' as lam^4, so
    halving lam divides the residual by about 2^12, and it stays far below the shift."""
    m = sy.molecule(8, 2, 10, 25)
    for p in (1, 2):                                # highest occupied, lowest empty
        res = []
        for lam in (0.4, 0.2):
            r = qsgw.g0w0_pass(lam * m["L"], m["eps"], m["C"], 2, ETA)
            wq = r["eps_qp"][p]
            s = qsgw.sigma_c_at(r["w"], m["eps"], r["Omega"], 2, ETA, wq)[p, p]
            res.append(abs(wq - m["eps"][p] - s))
            assert res[-1] < 1e-4 * abs(wq - m["eps"][p])
        assert 2.0 ** 9 < res[0] / res[1] < 2.0 ** 13


def test_large_eta_returns_the_input():
    """Sigma_c falls as 1/eta^2: the QP shift of an HF start goes to zero and Z to 1."""
    m = sy.molecule(8, 2, 10, 26)
    shift = []
    for eta in (1e6, 1e7):
        r = qsgw.g0w0_pass(m["L"], m["eps"], m["C"], 2, eta)
        shift.append(np.max(np.abs(r["eps_qp"] - m["eps"])))
        assert np.max(np.abs(r["Z"] - 1.0)) < 1e-9
    assert shift[0] < 1e-8 and 50.0 < shift[0] / shift[1] < 200.0


def test_golden_regression():
    """The oracle still reproduces the stored small-workload values (tests/golden)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "qsmp2_g0w0_nb24_no5_na72_seed0.json")
    doc = json.load(open(path))
    w = doc["workload"]
    m = sy.molecule(w["n_basis"], w["n_occ"], w["n_aux"], w["seed"])
    r = qsgw.g0w0_pass(m["L"], m["eps"], m["C"], w["n_occ"], w["eta"])
    np.testing.assert_allclose(r["eps_qp"], doc["g0w0_eps_qp"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["Z"], doc["g0w0_z"], rtol=1e-12, atol=1e-12)
