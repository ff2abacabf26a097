"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake in the oracle (``oracle.qsgw``) for the length
of the test -- a dropped factor, a flipped sign, a wrong index range or ordering,
a transposed product -- and runs the pin checks of the ``test_oracle_*`` modules
(never the stored golden values, which the oracle itself wrote).  At least one pin
must fail with an assertion (or the oracle's own RPA-instability guard).  The
unmutated oracle passes every pin in the same list.

The mistakes are planted by replacing module attributes, so every caller inside
the oracle (``qsgw_pass``, ``qsmp2_pass``, ``g0w0_pass``, ``qsgw_pass_open``)
sees the mutated step while ``oracle.brute`` stays untouched.
"""
import numpy as np
import pytest

import test_oracle_g0w0 as TG
import test_oracle_mp2 as TM
import test_oracle_open_shell as TO
import test_oracle_pins as TP
from oracle import qsgw

PINS = [
    ("two_level", lambda: TP.test_two_level_closed_form({})),
    ("two_level_strong", lambda: TP.test_two_level_closed_form(dict(e0=-3.0, e1=1.5, b=0.9))),
    ("casida_brute", lambda: TP.test_casida_spin_orbital_brute_force(11, 6, 2, 5)),
    ("residues_brute", lambda: TP.test_residues_spin_orbital_brute_force(21, 6, 2, 5)),
    ("sum_rules", TP.test_sum_rules),
    ("symmetry", TP.test_sigma_symmetry),
    ("ao_rotation", TP.test_ao_rotation_invariance),
    ("mo_sign", TP.test_mo_sign_covariance),
    ("weak_coupling_mp2", TP.test_weak_coupling_mp2_direct_limit),
    ("weak_coupling_freq", TP.test_weak_coupling_first_order_frequencies),
    ("four_index", TP.test_exchange_and_hartree_four_index),
    ("hf_fixed_point", TP.test_hf_fixed_point_exchange_only),
    ("large_eta", TP.test_large_eta_kills_correlation),
    ("loops_jacobi", lambda: TP.test_loops_and_jacobi(84, 6, 2, 12)),
    ("degenerate", TP.test_degenerate_energies_projector),
    ("orthonormal", TP.test_iterations_keep_orthonormal_orbitals),
    ("h_ao_fixed", TP.test_core_hamiltonian_fixed_in_ao_basis),
    ("mp2_two_level", lambda: TM.test_two_level_closed_form((-0.7, 0.4, 0.3, -0.2, 0.25))),
    ("mp2_spin_orbital", lambda: TM.test_spin_orbital_expansion(3, 6, 2, 5)),
    ("mp2_direct", TM.test_direct_term_matches_brute_force),
    ("mp2_rows", TM.test_rows_are_sigma_at_each_row_energy),
    ("mp2_symmetry", TM.test_sigma_symmetric_at_fixed_frequency),
    ("mp2_scaling", TM.test_fourth_power_scaling_and_ao_rotation),
    ("mp2_fixed_point", TM.test_qsmp2_fixed_point_without_correlation_strength),
    ("g0w0_two_level", lambda: TG.test_two_level_closed_form((-0.7, 0.4, 0.3, -0.2, 0.25))),
    ("g0w0_loops", lambda: TG.test_diagonal_matches_brute_force_loops(21, 6, 2, 5)),
    ("g0w0_slope", TG.test_derivative_is_the_slope_of_sigma),
    ("g0w0_hf_start", TG.test_hf_start_and_explicit_h_agree),
    ("g0w0_second_order", TG.test_linearised_energy_solves_the_qp_equation_to_second_order),
    ("g0w0_large_eta", TG.test_large_eta_returns_the_input),
    ("open_closed_limit", TO.test_closed_shell_limit),
    ("open_casida_brute", lambda: TO.test_spin_orbital_casida_brute_force(32, 6, (2, 1), 5)),
    ("open_one_electron", TO.test_one_electron_two_levels),
    ("open_spin_swap", TO.test_spin_swap_symmetry),
    ("open_hf_fixed_point", TO.test_hf_fixed_point_per_spin),
]


# --------------------------------------------------------------------------
# Mutants: each returns {attribute of oracle.qsgw: replacement}
# --------------------------------------------------------------------------
_orig = {k: getattr(qsgw, k) for k in dir(qsgw) if callable(getattr(qsgw, k))}


def _ri_transposed():
    def ri_mo_transform(L, C):                       # C L C^T instead of C^T L C
        return np.stack([C @ L[P] @ C.T for P in range(L.shape[0])])
    return {"ri_mo_transform": ri_mo_transform}


def _casida_kernel(factor, sign=1.0):
    def casida_AB(B, eps, n_occ):
        i, a = qsgw.transitions(eps.shape[0], n_occ)
        D = eps[a] - eps[i]
        K = B[:, i, a].T @ B[:, i, a]
        return np.diag(D) + sign * factor * K, sign * factor * K, D
    return {"casida_AB": casida_AB}


def _casida_M_unsymmetrised():
    def casida_M(A, Bc, D):                          # (A - B)(A + B), not its symmetric form
        return D[:, None] * (A + Bc)
    return {"casida_M": casida_M}


def _casida_M_difference():
    def casida_M(A, Bc, D):                          # A - B in the middle
        sq = np.sqrt(D)
        return sq[:, None] * (A - Bc) * sq[None, :]
    return {"casida_M": casida_M}


def _rpa_xpy(spin=np.sqrt(2.0), om_pow=-0.5, d_pow=0.5, sqrt_lam=True):
    def rpa_eigensolve(M, D):
        lam, Z = np.linalg.eigh(M)
        if lam[0] <= 0.0:
            raise FloatingPointError("RPA instability")
        Z = qsgw.fix_gauge(Z)
        Om = np.sqrt(lam) if sqrt_lam else lam
        return Om, spin * D[:, None] ** d_pow * Z * Om[None, :] ** om_pow, Z
    return {"rpa_eigensolve": rpa_eigensolve}


def _residues_virtual_major():
    def gw_residues(B, XpY, n_occ):                  # R's transitions in a-major order
        nb = B.shape[1]
        nv = nb - n_occ
        i = np.tile(np.arange(n_occ), nv)
        a = np.repeat(np.arange(n_occ, nb), n_occ)
        R = B[:, i, a] @ XpY
        return R, np.einsum("Ppq,Ps->spq", B, R)
    return {"gw_residues": gw_residues}


def _sigma_x(scale=-1.0, all_orbitals=False):
    def sigma_x(B, n_occ):
        Bo = B if all_orbitals else B[:, :, :n_occ]
        return scale * np.einsum("Ppi,Pqi->pq", Bo, Bo)
    return {"sigma_x": sigma_x}


def _hartree(scale=2.0, upper=0):
    def hartree(B, n_occ):
        k = n_occ + upper
        rho = np.einsum("Pii->P", B[:, :k, :k])
        return scale * np.einsum("Ppq,P->pq", B, rho)
    return {"hartree": hartree}


def _g_real(kind):
    def g_real(x, eta):
        if kind == "eta_unsquared":
            return x / (x * x + eta)
        if kind == "minus":
            return x / (x * x - eta * eta)
        return -x / (x * x + eta * eta)
    return {"g_real": g_real}


def _sigma_c_rows(kind):
    def sigma_c_rows(w, eps, Omega, n_occ, eta):
        nb = eps.shape[0]
        S = np.zeros((nb, nb))
        for m in range(nb):
            occ = m <= n_occ if kind == "boundary" else m < n_occ
            if kind == "shift_swapped":
                occ = not occ
            shift = Omega if occ else -Omega
            x = eps[:, None] - eps[m] + shift[None, :]
            if kind == "frequency_sign":
                x = eps[m] - eps[:, None] + shift[None, :]
            wm = w[:, :, m].T
            S += (wm * qsgw.g_real(x, eta)) @ wm.T
        return S
    return {"sigma_c_rows": sigma_c_rows}


def _sigma_c_qs_unsymmetrised():
    return {"sigma_c_qs": lambda S: S.copy()}


def _qs_update(kind):
    def qs_update(h_mo, J, Sx, Sc, C):
        H = h_mo + J + Sc + (0.0 if kind == "no_exchange" else Sx)
        H = 0.5 * (H + H.T)
        e, U = np.linalg.eigh(H)
        U = qsgw.fix_gauge(U)
        Cn = {"left": U @ C, "bare": U}.get(kind, C @ U)
        hn = U @ h_mo @ U.T if kind == "h_transposed" else U.T @ h_mo @ U
        return e, Cn, hn, U
    return {"qs_update": qs_update}


def _hf_core_plus_exchange():
    def hf_core_mo(B, eps, n_occ):
        return np.diag(eps) - qsgw.hartree(B, n_occ) + qsgw.sigma_x(B, n_occ)
    return {"hf_core_mo": hf_core_mo}


def _mp2_factors_exchange(kind):
    def mp2_factors(B, n_occ, p):
        na, nb = B.shape[0], B.shape[1]
        nv = nb - n_occ
        i, a = qsgw.transitions(nb, n_occ)
        Ap = B[:, :, p].T @ B[:, i, a]
        printed = (kind == "printed") or (kind == "swapped" and p >= n_occ)
        occ_form = (p < n_occ) != (kind == "swapped")
        if occ_form and not printed:
            X = B[:, p, n_occ:].T @ B[:, :n_occ, :].reshape(na, n_occ * nb)   # (p a|i n)
            Xp = X.reshape(nv, n_occ, nb).transpose(2, 1, 0)
        else:
            X = B[:, p, :n_occ].T @ B[:, n_occ:, :].reshape(na, nv * nb)      # (p i|a n)
            Xp = X.reshape(n_occ, nv, nb).transpose(2, 0, 1)
        return Ap, Xp.reshape(nb, n_occ * nv)
    return {"mp2_factors": mp2_factors}


def _mp2_sums(direct=2.0, occ_sign=1.0):
    def terms(B, eps, n_occ, eta, x_of):
        nb = eps.shape[0]
        i, a = qsgw.transitions(nb, n_occ)
        D = eps[a] - eps[i]
        out = np.zeros((nb, nb))
        for p in range(nb):
            Ap, Xp = qsgw.mp2_factors(B, n_occ, p)
            sgn = occ_sign if p < n_occ else -1.0
            out += (Ap * qsgw.g_real(x_of(p, sgn * D), eta)) @ (direct * Ap - Xp).T
        return out

    def sigma_mp2_at(B, eps, n_occ, eta, omega):
        return terms(B, eps, n_occ, eta, lambda p, sD: omega - eps[p] + sD[None, :])

    def sigma_mp2_rows(B, eps, n_occ, eta):
        return terms(B, eps, n_occ, eta, lambda p, sD: eps[:, None] - eps[p] + sD[None, :])
    return {"sigma_mp2_at": sigma_mp2_at, "sigma_mp2_rows": sigma_mp2_rows}


def _g_derivative_sign():
    def g_real_derivative(x, eta):
        d = x * x + eta * eta
        return (x * x - eta * eta) / (d * d)
    return {"g_real_derivative": g_real_derivative}


def _g0w0(kind):
    def g0w0_pass(L, eps, C, n_occ, eta, h_mo=None):
        B = qsgw.ri_mo_transform(L, C)
        J = qsgw.hartree(B, n_occ)
        Sx = qsgw.sigma_x(B, n_occ)
        if h_mo is None:
            h_mo = qsgw.hf_core_mo(B, eps, n_occ)
        A, Bc, D = qsgw.casida_AB(B, eps, n_occ)
        Omega, XpY, _ = qsgw.rpa_eigensolve(qsgw.casida_M(A, Bc, D), D)
        _, w = qsgw.gw_residues(B, XpY, n_occ)
        sig, dsig = qsgw.sigma_c_diag(w, eps, Omega, n_occ, eta)
        v = eps - np.diag(h_mo) + (np.diag(J) if kind == "v_sign" else -np.diag(J))
        Z = 1.0 / (1.0 + dsig) if kind == "z_sign" else 1.0 / (1.0 - dsig)
        eqp = eps + (1.0 if kind == "no_z" else Z) * (np.diag(Sx) + sig - v)
        return {"Omega": Omega, "w": w, "sigma_c_diag": sig, "dsigma_c_diag": dsig, "Z": Z,
                "eps_qp": eqp, "sigma_x_diag": np.diag(Sx).copy(), "v_diag": v}
    return {"g0w0_pass": g0w0_pass}


def _sigma_c_diag_shift_swapped():
    def sigma_c_diag(w, eps, Omega, n_occ, eta):
        sig, dsig = np.zeros(eps.shape[0]), np.zeros(eps.shape[0])
        for m in range(eps.shape[0]):
            shift = -Omega if m < n_occ else Omega
            x = eps[:, None] - eps[m] + shift[None, :]
            w2 = w[:, :, m].T ** 2
            sig += np.sum(w2 * qsgw.g_real(x, eta), axis=1)
            dsig += np.sum(w2 * qsgw.g_real_derivative(x, eta), axis=1)
        return sig, dsig
    return {"sigma_c_diag": sigma_c_diag}


def _casida_open_factor(f):
    def casida_M_open(Bs, epss, n_occs):
        Dl, Bl = [], []
        for B, eps, no in zip(Bs, epss, n_occs):
            i, a = qsgw.transitions(eps.shape[0], no)
            Dl.append(eps[a] - eps[i])
            Bl.append(B[:, i, a])
        D, Bt = np.concatenate(Dl), np.concatenate(Bl, axis=1)
        sq = np.sqrt(D)
        return np.diag(D * D) + f * sq[:, None] * (Bt.T @ Bt) * sq[None, :], D, Bt
    return {"casida_M_open": casida_M_open}


def _rpa_open_spin_factor():
    def rpa_eigensolve_open(M, D):
        Om, XpY, Z = _orig["rpa_eigensolve_open"](M, D)
        return Om, np.sqrt(2.0) * XpY, Z
    return {"rpa_eigensolve_open": rpa_eigensolve_open}


def _hartree_open(kind):
    def hartree_open(B, Bs, n_occs):
        if kind == "factor2":
            return 2.0 * _orig["hartree_open"](B, Bs, n_occs)
        # own-spin density taken as a closed shell: 2 sum_{i in own occ}
        k = [Bx is B for Bx in Bs].index(True) if any(Bx is B for Bx in Bs) else 0
        return qsgw.hartree(B, n_occs[k])
    return {"hartree_open": hartree_open}


MUTANTS = {
    "ri_transposed": _ri_transposed,
    "kernel_spin_sum_dropped": lambda: _casida_kernel(1.0),
    "kernel_sign_flipped": lambda: _casida_kernel(2.0, -1.0),
    "kernel_factor_four": lambda: _casida_kernel(4.0),
    "M_unsymmetrised": _casida_M_unsymmetrised,
    "M_with_A_minus_B": _casida_M_difference,
    "xpy_no_sqrt2": lambda: _rpa_xpy(spin=1.0),
    "xpy_omega_power": lambda: _rpa_xpy(om_pow=0.5),
    "xpy_no_sqrt_d": lambda: _rpa_xpy(d_pow=0.0),
    "omega_not_square_root": lambda: _rpa_xpy(sqrt_lam=False),
    "residues_virtual_major": _residues_virtual_major,
    "sigma_x_all_orbitals": lambda: _sigma_x(all_orbitals=True),
    "sigma_x_factor_two": lambda: _sigma_x(scale=-2.0),
    "sigma_x_sign": lambda: _sigma_x(scale=1.0),
    "hartree_no_spin_sum": lambda: _hartree(scale=1.0),
    "hartree_one_orbital_too_many": lambda: _hartree(upper=1),
    "g_eta_unsquared": lambda: _g_real("eta_unsquared"),
    "g_minus_eta_squared": lambda: _g_real("minus"),
    "g_sign": lambda: _g_real("sign"),
    "sigma_c_shift_swapped": lambda: _sigma_c_rows("shift_swapped"),
    "sigma_c_occupied_boundary": lambda: _sigma_c_rows("boundary"),
    "sigma_c_frequency_sign": lambda: _sigma_c_rows("frequency_sign"),
    "sigma_c_not_hermitised": _sigma_c_qs_unsymmetrised,
    "H_without_exchange": lambda: _qs_update("no_exchange"),
    "C_new_left_product": lambda: _qs_update("left"),
    "C_new_without_C": lambda: _qs_update("bare"),
    "h_new_transposed_rotation": lambda: _qs_update("h_transposed"),
    "hf_core_exchange_sign": _hf_core_plus_exchange,
    "mp2_printed_exchange": lambda: _mp2_factors_exchange("printed"),
    "mp2_exchange_forms_swapped": lambda: _mp2_factors_exchange("swapped"),
    "mp2_direct_factor_one": lambda: _mp2_sums(direct=1.0),
    "mp2_occupied_denominator_sign": lambda: _mp2_sums(occ_sign=-1.0),
    "g0w0_derivative_sign": _g_derivative_sign,
    "g0w0_z_sign": lambda: _g0w0("z_sign"),
    "g0w0_no_renormalisation": lambda: _g0w0("no_z"),
    "g0w0_potential_hartree_sign": lambda: _g0w0("v_sign"),
    "g0w0_diag_shift_swapped": _sigma_c_diag_shift_swapped,
    "open_kernel_closed_shell_factor": lambda: _casida_open_factor(4.0),
    "open_kernel_one": lambda: _casida_open_factor(1.0),
    "open_xpy_sqrt2": _rpa_open_spin_factor,
    "open_hartree_factor_two": lambda: _hartree_open("factor2"),
    "open_hartree_own_spin_closed": lambda: _hartree_open("own"),
}


def _first_failing_pin():
    for name, check in PINS:
        try:
            check()
        except (AssertionError, FloatingPointError):
            return name
    return None


def test_unmutated_oracle_passes_every_pin():
    assert _first_failing_pin() is None


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_mutant_is_caught(mutant, monkeypatch):
    for attr, fn in MUTANTS[mutant]().items():
        assert hasattr(qsgw, attr), attr
        monkeypatch.setattr(qsgw, attr, fn)
    caught = _first_failing_pin()
    assert caught is not None, f"no pin fails with the mistake {mutant!r} planted in the oracle"
