"""Pins of the CPU oracle against what the paper's equations and mathematics fix.

Each test checks the oracle (``oracle.qsgw``) against something other than
itself: a closed form, a brute-force form of the same equation with every index
written out (``oracle.brute``), an invariance, a sum rule or a limit.  The
paper prints no worked example, so there are no printed values to compare with.
"""
import math

import numpy as np
import pytest

import synthetic as sy
from oracle import brute, qsgw

ETA = 1e-3


def tiny(seed=11, nb=6, no=2, na=5):
    return sy.molecule(nb, no, na, seed)


# --------------------------------------------------------------------------
# P1: two-level model (nb = 2, no = 1, na = 1) in closed form
# --------------------------------------------------------------------------
def two_level(e0=-0.7, e1=0.4, b00=0.3, b11=-0.2, b=0.25):
    """A single aux function with MO-basis factor [[b00, b], [b, b11]] (C = I)."""
    L = np.array([[[b00, b], [b, b11]]])
    eps = np.array([e0, e1])
    return L, eps, np.eye(2)


@pytest.mark.parametrize("params", [dict(), dict(e0=-3.0, e1=1.5, b=0.9), dict(b=1e-3)])
def test_two_level_closed_form(params):
    L, eps, C = two_level(**params)
    b00, b, b11 = L[0, 0, 0], L[0, 0, 1], L[0, 1, 1]
    delta = eps[1] - eps[0]
    eta = 1e-3
    r = qsgw.qsgw_pass(L, eps, C, 1, eta)
    # Casida 2x2: [[d + 2b^2, 2b^2], [-2b^2, -d - 2b^2]] -> Omega^2 = d^2 + 4 d b^2
    Om = math.sqrt(delta * delta + 4.0 * delta * b * b)
    assert r["Omega"][0] == pytest.approx(Om, rel=1e-14)
    # (X+Y) = sqrt(2) sqrt(d / Omega); w_pq = B_pq * b * (X+Y)
    xpy = math.sqrt(2.0 * delta / Om)
    assert abs(r["XpY"][0, 0]) == pytest.approx(xpy, rel=1e-14)
    w = np.array([[b00, b], [b, b11]]) * b * xpy
    np.testing.assert_allclose(np.abs(r["w"][0]), np.abs(w), rtol=1e-13)
    g = lambda x: x / (x * x + eta * eta)
    S = np.zeros((2, 2))
    for p in range(2):
        for q in range(2):
            S[p, q] = w[p, 0] * w[q, 0] * g(eps[p] - eps[0] + Om) + w[p, 1] * w[q, 1] * g(eps[p] - eps[1] - Om)
    np.testing.assert_allclose(r["sigma_c"], 0.5 * (S + S.T), rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(r["sigma_x"], -np.outer([b00, b], [b00, b]), rtol=1e-14)
    J = 2.0 * b00 * np.array([[b00, b], [b, b11]])
    np.testing.assert_allclose(r["J"], J, rtol=1e-14)
    # HF-consistent h: h + J + Sx = diag(eps); the 2x2 QP Hamiltonian in closed form
    H = np.diag(eps) + r["sigma_c"]
    tr, det = H[0, 0] + H[1, 1], H[0, 0] * H[1, 1] - H[0, 1] ** 2
    disc = math.sqrt(max(tr * tr / 4 - det, 0.0))
    np.testing.assert_allclose(r["eps_new"], [tr / 2 - disc, tr / 2 + disc], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("params", [dict(), dict(e0=-3.0, e1=1.5, b=0.9)])
def test_two_level_closed_form_streamed_residues(params):
    """The same closed form through the path that forms the residues of one orbital m
    at a time (keep_w=False, used for the large stored workloads)."""
    L, eps, C = two_level(**params)
    b00, b, b11 = L[0, 0, 0], L[0, 0, 1], L[0, 1, 1]
    delta = eps[1] - eps[0]
    eta = 1e-3
    r = qsgw.qsgw_pass(L, eps, C, 1, eta, keep_w=False)
    assert r["w"] is None
    Om = math.sqrt(delta * delta + 4.0 * delta * b * b)
    w = np.array([[b00, b], [b, b11]]) * b * math.sqrt(2.0 * delta / Om)
    g = lambda x: x / (x * x + eta * eta)
    S = np.zeros((2, 2))
    for p in range(2):
        for q in range(2):
            S[p, q] = w[p, 0] * w[q, 0] * g(eps[p] - eps[0] + Om) + w[p, 1] * w[q, 1] * g(eps[p] - eps[1] - Om)
    np.testing.assert_allclose(r["sigma_c"], 0.5 * (S + S.T), rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("seed,nb,no,na", [(91, 6, 2, 5), (92, 9, 4, 20), (93, 7, 1, 3)])
def test_streamed_residues_match_index_loops(seed, nb, no, na):
    """Sigma_c with per-orbital residues equals four nested loops over (p, q, m, s) of
    Eq. (Sigma.c.GW) on the full residues, and the residues of one orbital are the
    slice w[:, :, m] of Eq. (w.residue)."""
    m = tiny(seed, nb, no, na)
    full = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, ETA)
    lean = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, ETA, keep_w=False)
    S_loop = brute.sigma_c_loops(full["w"], m["eps"], full["Omega"], no, ETA)
    np.testing.assert_allclose(lean["sigma_c"], 0.5 * (S_loop + S_loop.T),
                               atol=1e-12 * max(1.0, np.abs(S_loop).max()))
    for k in range(nb):
        np.testing.assert_allclose(qsgw.residues_of_state(full["B"], lean["R"], k), full["w"][:, :, k].T,
                                   atol=1e-14)
    np.testing.assert_allclose(lean["eps_new"], full["eps_new"], atol=1e-12)


@pytest.mark.parametrize("seed,nb,no,na", [(95, 9, 4, 20), (96, 12, 3, 7)])
def test_casida_operator_equals_the_formed_matrix(seed, nb, no, na):
    """The matrix-free product M x (used for the largest workload) equals the formed
    M of Eq. (Casida.AB.XY) times x, whose eigenvalues the brute-force Casida pin fixes."""
    m = tiny(seed, nb, no, na)
    B = qsgw.ri_mo_transform(m["L"], m["C"])
    A, Bc, D = qsgw.casida_AB(B, m["eps"], no)
    M = qsgw.casida_M(A, Bc, D)
    apply, D2 = qsgw.casida_M_apply(B, m["eps"], no)
    np.testing.assert_array_equal(D2, D)
    x = np.random.default_rng(seed).standard_normal((D.shape[0], 3))
    np.testing.assert_allclose(apply(x), M @ x, rtol=1e-12, atol=1e-13 * np.abs(M).max())
    np.testing.assert_allclose(apply(x[:, 0]), M @ x[:, 0], rtol=1e-12, atol=1e-13 * np.abs(M).max())
    lam = np.linalg.eigvalsh(np.column_stack([apply(e) for e in np.eye(D.shape[0])]))
    assert np.sum(lam) == pytest.approx(np.trace(M), rel=1e-12)
    np.testing.assert_allclose(np.sqrt(lam), qsgw.rpa_eigensolve(M, D)[0], rtol=1e-12)


# --------------------------------------------------------------------------
# P2: brute-force non-Hermitian Casida over spin orbitals
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed,nb,no,na", [(11, 6, 2, 5), (12, 5, 1, 3), (13, 6, 3, 8), (14, 4, 3, 2)])
def test_casida_spin_orbital_brute_force(seed, nb, no, na):
    m = tiny(seed, nb, no, na)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, ETA)
    vals, _, _, _ = brute.casida_spin_orbital(m["L"], m["C"], m["eps"], no)
    n_ov = no * (nb - no)
    # eigenvalues come in +/- pairs: singlets +/-Omega_s and spin-flip +/-D_t
    expect = np.sort(np.concatenate([r["Omega"], r["D"]]))
    np.testing.assert_allclose(np.sort(vals[vals > 0]), expect, rtol=1e-11)
    np.testing.assert_allclose(np.sort(-vals[vals < 0]), expect, rtol=1e-11)
    assert vals.shape[0] == 4 * n_ov


@pytest.mark.parametrize("seed,nb,no,na", [(21, 6, 2, 5), (22, 5, 2, 4)])
def test_residues_spin_orbital_brute_force(seed, nb, no, na):
    """Eq. (w.residue) with the sigma' sum written out fixes the sqrt(2) of reading R2."""
    m = tiny(seed, nb, no, na)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, ETA)
    Om, w, Otrip = brute.singlet_residues_spin_orbital(m["L"], m["C"], m["eps"], no)
    order = np.argsort(Om)
    Om, w = Om[order], w[order]
    np.testing.assert_allclose(Om, r["Omega"], rtol=1e-11)
    np.testing.assert_allclose(np.sort(Otrip), np.sort(r["D"]), rtol=1e-11)
    for s in range(Om.shape[0]):  # the residue sign is a gauge: compare w w^T
        np.testing.assert_allclose(np.outer(w[s], w[s]), np.outer(r["w"][s], r["w"][s]),
                                   rtol=1e-8, atol=1e-12)


# --------------------------------------------------------------------------
# P3: sum rules of the RPA eigenvectors
# --------------------------------------------------------------------------
def test_sum_rules():
    m = tiny(31, 8, 3, 10)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], 3, ETA)
    XpY, Om, D = r["XpY"], r["Omega"], r["D"]
    # sum_s Omega_s (X+Y)_ts (X+Y)_us = 2 D_t delta_tu
    np.testing.assert_allclose((XpY * Om[None, :]) @ XpY.T, 2.0 * np.diag(D), atol=1e-12)
    # (X+Y) Omega^-1 (X+Y)^T = 2 (A+B)^-1
    A, Bc, _ = qsgw.casida_AB(r["B"], m["eps"], 3)
    np.testing.assert_allclose((XpY / Om[None, :]) @ XpY.T, 2.0 * np.linalg.inv(A + Bc), atol=1e-12)
    # tr M = sum Omega^2
    assert np.trace(r["M"]) == pytest.approx(np.sum(Om ** 2), rel=1e-13)


# --------------------------------------------------------------------------
# P4: symmetry
# --------------------------------------------------------------------------
def test_sigma_symmetry():
    m = tiny(41, 9, 3, 12)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], 3, ETA)
    for key in ("sigma_x", "sigma_c", "J"):
        X = r[key]
        assert np.max(np.abs(X - X.T)) <= 1e-14 * np.max(np.abs(X))
    # Sigma_pq(omega) = Sigma_qp(omega) at any frequency
    Sw = qsgw.sigma_c_at(r["w"], m["eps"], r["Omega"], 3, ETA, 0.37)
    assert np.max(np.abs(Sw - Sw.T)) <= 1e-13 * np.max(np.abs(Sw))


# --------------------------------------------------------------------------
# P5: invariance under orthogonal rotation of the AO basis and MO sign flips
# --------------------------------------------------------------------------
def test_ao_rotation_invariance():
    m = tiny(51, 8, 3, 10)
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    L2 = np.einsum("mi,Pmn,nj->Pij", U, m["L"], U)     # U^T L^P U
    C2 = U.T @ m["C"]
    r1 = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], 3, ETA)
    r2 = qsgw.qsgw_pass(L2, m["eps"], C2, 3, ETA)
    np.testing.assert_allclose(r2["B"], r1["B"], atol=1e-13)
    np.testing.assert_allclose(r2["Omega"], r1["Omega"], rtol=1e-12)
    np.testing.assert_allclose(r2["sigma_c"], r1["sigma_c"], atol=1e-12 * np.abs(r1["sigma_c"]).max())
    np.testing.assert_allclose(r2["eps_new"], r1["eps_new"], atol=1e-12)


def test_mo_sign_covariance():
    m = tiny(52, 7, 2, 9)
    s = np.array([1, -1, -1, 1, -1, 1, 1.0])
    r1 = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], 2, ETA)
    r2 = qsgw.qsgw_pass(m["L"], m["eps"], m["C"] * s[None, :], 2, ETA)
    np.testing.assert_allclose(r2["Omega"], r1["Omega"], rtol=1e-12)
    np.testing.assert_allclose(r2["eps_new"], r1["eps_new"], atol=1e-12)
    ss = np.outer(s, s)
    for key in ("sigma_x", "sigma_c"):
        np.testing.assert_allclose(r2[key], ss * r1[key], atol=1e-12 * np.abs(r1[key]).max())


# --------------------------------------------------------------------------
# P6: weak coupling -> direct term of the MP2 self-energy (Eq. Sigma.c.MP2)
# --------------------------------------------------------------------------
def test_weak_coupling_mp2_direct_limit():
    m = tiny(61, 6, 2, 5)
    eta = 0.05   # keeps every denominator well away from a pole
    gaps = []
    for lam in (1e-1, 1e-2, 1e-3):
        L = m["L"] * lam
        r = qsgw.qsgw_pass(L, m["eps"], m["C"], 2, eta)
        g = brute.eri_mo(L, m["C"])
        # compare row p of Sigma at omega = eps_p
        Smp2 = np.array([brute.sigma_mp2_direct(g, m["eps"], 2, eta, m["eps"][p])[p] for p in range(6)])
        Sgw = qsgw.sigma_c_rows(r["w"], m["eps"], r["Omega"], 2, eta)
        gaps.append(np.max(np.abs(Sgw - Smp2)) / np.max(np.abs(Smp2)))
        # Omega_s -> D + 2 K_ss (first order in the kernel); corrections are O(lam^4)
    assert gaps[1] < 0.02 * gaps[0] and gaps[2] < 0.02 * gaps[1], gaps
    assert gaps[2] < 1e-4


def test_weak_coupling_first_order_frequencies():
    m = tiny(62, 6, 2, 5)
    errs = []
    for lam in (1e-1, 1e-2):
        L = m["L"] * lam
        B = qsgw.ri_mo_transform(L, m["C"])
        A, Bc, D = qsgw.casida_AB(B, m["eps"], 2)
        Om, _, _ = qsgw.rpa_eigensolve(qsgw.casida_M(A, Bc, D), D)
        errs.append(np.max(np.abs(Om - np.sort(np.diag(A)))) / lam ** 2)
    assert errs[1] < 0.05 * errs[0]


# --------------------------------------------------------------------------
# P7: exchange-only limit, Hartree and exchange from four-index integrals
# --------------------------------------------------------------------------
def test_exchange_and_hartree_four_index():
    m = tiny(71, 7, 3, 6)
    B = qsgw.ri_mo_transform(m["L"], m["C"])
    J4, Kx4 = brute.hartree_exchange_mo(m["L"], m["C"], 3)
    np.testing.assert_allclose(qsgw.hartree(B, 3), J4, atol=1e-13)
    np.testing.assert_allclose(qsgw.sigma_x(B, 3), Kx4, atol=1e-13)
    g = brute.eri_mo(m["L"], m["C"])
    np.testing.assert_allclose(np.einsum("Ppq,Prs->pqrs", B, B), g, atol=1e-13)


def test_hf_fixed_point_exchange_only():
    m = tiny(72, 8, 3, 9)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], 3, ETA, correlation=False)
    np.testing.assert_allclose(r["eps_new"], m["eps"], atol=1e-13)
    # C' spans the same orbitals: projector onto each MO is unchanged
    np.testing.assert_allclose(np.abs(np.sum(r["C_new"] * m["C"], axis=0)), 1.0, atol=1e-12)


def test_large_eta_kills_correlation():
    m = tiny(73, 6, 2, 5)
    S1 = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], 2, 1e4)["sigma_c"]
    S2 = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], 2, 1e5)["sigma_c"]
    # Sigma_c ~ 1/eta^2 for eta much larger than every denominator
    ratio = np.max(np.abs(S1)) / np.max(np.abs(S2))
    assert ratio == pytest.approx(100.0, rel=1e-3)


# --------------------------------------------------------------------------
# P8: brute force on small shapes
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed,nb,no,na", [(81, 5, 1, 4), (82, 6, 5, 3), (83, 7, 3, 1), (84, 6, 2, 12)])
def test_loops_and_jacobi(seed, nb, no, na):
    m = tiny(seed, nb, no, na)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, ETA)
    S_loop = brute.sigma_c_loops(r["w"], m["eps"], r["Omega"], no, ETA)
    S_mat = qsgw.sigma_c_rows(r["w"], m["eps"], r["Omega"], no, ETA)
    np.testing.assert_allclose(S_mat, S_loop, atol=1e-12 * max(1.0, np.abs(S_loop).max()))
    lam, Z = brute.jacobi_eigh(r["M"])
    np.testing.assert_allclose(np.sqrt(lam), r["Omega"], rtol=1e-12)
    H = r["h_mo"] + r["J"] + r["sigma_x"] + r["sigma_c"]
    e, _ = brute.jacobi_eigh(H)
    np.testing.assert_allclose(e, r["eps_new"], atol=1e-12)


def test_degenerate_energies_projector():
    """Degenerate virtual energies: the Omega set and Sigma stay well defined."""
    m = tiny(85, 6, 2, 5)
    eps = m["eps"].copy()
    eps[3] = eps[2]
    r = qsgw.qsgw_pass(m["L"], eps, m["C"], 2, ETA)
    vals, _, _, _ = brute.casida_spin_orbital(m["L"], m["C"], eps, 2)
    np.testing.assert_allclose(np.sort(vals[vals > 0]), np.sort(np.concatenate([r["Omega"], r["D"]])), rtol=1e-10)


def test_rpa_instability_detected():
    """With the opposite Coulomb sign M can lose positivity; the oracle refuses it."""
    D = np.array([0.1, 0.2])
    M = np.diag(D * D) - 0.5 * np.ones((2, 2))
    with pytest.raises(FloatingPointError):
        qsgw.rpa_eigensolve(M, D)


def test_iterations_keep_orthonormal_orbitals():
    m = tiny(91, 8, 3, 10)
    its = qsgw.qsgw_iterations(m["L"], m["eps"], m["C"], 3, ETA, 3)
    for r in its:
        C = r["C_new"]
        np.testing.assert_allclose(C.T @ C, np.eye(8), atol=1e-13)
        assert np.all(np.diff(r["eps_new"]) >= 0)


def test_core_hamiltonian_fixed_in_ao_basis():
    """Eq. (H) with S = I: h is one fixed operator on the AO basis, so C h_MO C^T is the same
    before and after every iteration, and H = h + J + Sigma_x + Sigma_c, carried to the AO
    basis by the input orbitals, is diagonal in the updated ones: C'^T H_AO C' = diag(eps')."""
    m = tiny(92, 8, 3, 10)
    its = qsgw.qsgw_iterations(m["L"], m["eps"], m["C"], 3, ETA, 2)
    C = m["C"]
    h_ao = C @ its[0]["h_mo"] @ C.T
    for r in its:
        H_ao = C @ (r["h_mo"] + r["J"] + r["sigma_x"] + r["sigma_c"]) @ C.T
        Cn = r["C_new"]
        np.testing.assert_allclose(Cn.T @ H_ao @ Cn, np.diag(r["eps_new"]), atol=1e-13)
        np.testing.assert_allclose(Cn @ r["h_mo_new"] @ Cn.T, h_ao, atol=1e-13)
        C = Cn


def test_golden_regression():
    """The oracle still reproduces the stored small-workload values (tests/golden)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "qsgw_nb24_no5_na72_seed0.json")
    doc = json.load(open(path))
    w = doc["workload"]
    m = sy.molecule(w["n_basis"], w["n_occ"], w["n_aux"], w["seed"])
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], w["n_occ"], w["eta"])
    np.testing.assert_allclose(r["Omega"], doc["Omega"], rtol=1e-12)
    np.testing.assert_allclose(r["eps_new"], doc["eps_new"], atol=1e-12)
    np.testing.assert_allclose(r["sigma_c"], doc["sigma_c"], atol=1e-12)
    np.testing.assert_allclose(r["sigma_x"], doc["sigma_x"], atol=1e-12)
