"""Pins of the open-shell (sigma-resolved) qsGW oracle, ``oracle.qsgw.qsgw_pass_open``."""
import math

import numpy as np
import pytest

import synthetic as sy
from oracle import brute, qsgw

ETA = 1e-3


def g_re(x, eta=ETA):
    return x / (x * x + eta * eta)


def test_closed_shell_limit():
    """Equal spin channels reproduce the closed-shell pass: the same Sigma_x, Sigma_c and
    quasiparticle energies per spin; the Casida frequencies are the closed-shell
    (singlet) ones plus the spin-flip combinations at Omega = D."""
    nb, no, na = 10, 3, 14
    m = sy.molecule(nb, no, na, 31)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, ETA)
    o = qsgw.qsgw_pass_open(m["L"], (m["eps"], m["eps"]), (m["C"], m["C"]), (no, no), ETA)
    want = np.sort(np.concatenate([r["Omega"], r["D"]]))
    np.testing.assert_allclose(o["Omega"], want, rtol=1e-10)
    for sp in o["spin"]:
        np.testing.assert_allclose(sp["sigma_x"], r["sigma_x"], rtol=1e-12, atol=1e-14)
        assert np.max(np.abs(sp["sigma_c"] - r["sigma_c"])) <= 1e-9 * np.max(np.abs(r["sigma_c"]))
        np.testing.assert_allclose(sp["J"], r["J"], rtol=1e-12, atol=1e-14)
        assert np.max(np.abs(sp["eps_new"] - r["eps_new"])) < 1e-9


@pytest.mark.parametrize("seed,nb,nos,na", [(32, 6, (2, 1), 5), (33, 5, (1, 0), 4), (34, 6, (3, 2), 7)])
def test_spin_orbital_casida_brute_force(seed, nb, nos, na):
    """The positive roots of the full spin-orbital Casida problem with one set of MOs per
    spin are the oracle's Omega."""
    m = sy.molecule(nb, nos[0], na, seed)
    rng = np.random.default_rng(seed)
    Cdn, _ = np.linalg.qr(rng.standard_normal((nb, nb)))
    edn = np.sort(m["eps"] + 0.1 * rng.standard_normal(nb))
    Cs, epss = (m["C"], Cdn), (m["eps"], edn)
    o = qsgw.qsgw_pass_open(m["L"], epss, Cs, nos, ETA)
    vals = brute.casida_spin_orbital_open(m["L"], Cs, epss, nos)
    pos = vals[vals > 0]
    np.testing.assert_allclose(pos, o["Omega"], rtol=1e-9)


def test_one_electron_two_levels():
    """nb = 2, one spin-up electron, one aux function, C = I: one transition (up 0 -> 1),
    Omega = sqrt(d^2 + 2 d b^2), X + Y = sqrt(d / Omega), w_pq = B_pq b sqrt(d / Omega) for
    both spins; spin down has no occupied orbital, no exchange, and only the 2p1h sum."""
    e_up, e_dn = np.array([-0.7, 0.4]), np.array([-0.2, 0.9])
    b00, b, b11 = 0.3, 0.25, -0.2
    L = np.array([[[b00, b], [b, b11]]])
    o = qsgw.qsgw_pass_open(L, (e_up, e_dn), (np.eye(2), np.eye(2)), (1, 0), ETA)
    d = e_up[1] - e_up[0]
    Om = math.sqrt(d * d + 2.0 * d * b * b)
    assert o["Omega"][0] == pytest.approx(Om, rel=1e-14)
    Bm = np.array([[b00, b], [b, b11]])
    w = Bm * b * math.sqrt(d / Om)
    S_up = np.array([[w[p, 0] * w[q, 0] * g_re(e_up[p] - e_up[0] + Om) + w[p, 1] * w[q, 1] * g_re(e_up[p] - e_up[1] - Om)
                      for q in range(2)] for p in range(2)])
    S_dn = np.array([[sum(w[p, mm] * w[q, mm] * g_re(e_dn[p] - e_dn[mm] - Om) for mm in range(2))
                      for q in range(2)] for p in range(2)])
    up, dn = o["spin"]
    np.testing.assert_allclose(up["sigma_c"], 0.5 * (S_up + S_up.T), rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(dn["sigma_c"], 0.5 * (S_dn + S_dn.T), rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(up["sigma_x"], -np.outer(Bm[:, 0], Bm[:, 0]), rtol=1e-14)
    assert np.all(dn["sigma_x"] == 0.0)
    np.testing.assert_allclose(up["J"], b00 * Bm, rtol=1e-14)
    np.testing.assert_allclose(dn["J"], b00 * Bm, rtol=1e-14)


def test_spin_swap_symmetry():
    nb, na = 8, 10
    m = sy.molecule(nb, 3, na, 35)
    rng = np.random.default_rng(1)
    Cdn, _ = np.linalg.qr(rng.standard_normal((nb, nb)))
    edn = np.sort(m["eps"] + 0.2 * rng.standard_normal(nb))
    a = qsgw.qsgw_pass_open(m["L"], (m["eps"], edn), (m["C"], Cdn), (3, 2), ETA)
    b = qsgw.qsgw_pass_open(m["L"], (edn, m["eps"]), (Cdn, m["C"]), (2, 3), ETA)
    np.testing.assert_allclose(a["Omega"], b["Omega"], rtol=1e-12)
    for k in (0, 1):
        np.testing.assert_allclose(a["spin"][k]["eps_new"], b["spin"][1 - k]["eps_new"], rtol=0, atol=1e-9)


def test_hf_fixed_point_per_spin():
    """With the correlation made negligible (eta -> large), each spin's update returns its
    input energies (reading R5 per spin)."""
    nb, na = 8, 10
    m = sy.molecule(nb, 3, na, 36)
    rng = np.random.default_rng(2)
    Cdn, _ = np.linalg.qr(rng.standard_normal((nb, nb)))
    edn = np.sort(m["eps"] + 0.2 * rng.standard_normal(nb))
    o = qsgw.qsgw_pass_open(m["L"], (m["eps"], edn), (m["C"], Cdn), (3, 2), 1e8)
    assert np.max(np.abs(o["spin"][0]["eps_new"] - m["eps"])) < 1e-9
    assert np.max(np.abs(o["spin"][1]["eps_new"] - edn)) < 1e-9
