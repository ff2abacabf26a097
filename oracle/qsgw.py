"""Plain CPU float64 oracle for one closed-shell RI-qsGW pass.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA library and never calls it.

Each function follows one equation of the paper (arXiv 2210.17093, Sec. II) in
the paper's order and notation, in float64 NumPy.  ``numpy.linalg.eigh`` and
matrix products serve as library steps; there is no blocking or fusion beyond
what the equations state.

Notation (closed shell, real orbitals, S = I):
  nb = n_basis, no = n_occ, nv = nb - no, n_ov = no*nv, na = n_aux;
  i, j occupied; a, b virtual; p, q, m any MO; P auxiliary; s excitation;
  transition index t = i*nv + (a - no) (occupied-major).

Readings taken where the paper is silent or ambiguous (each one is listed in
the design notes with its justification):
  R1  Coulomb kernel sign in Eqs. (Casida.A/B): "+" (standard RPA), so for
      singlets A = D + 2K, B = 2K with K_tu = (t|u).
  R2  The spin sum over sigma' in Eq. (w.residue) for a closed shell contributes
      sqrt(2), folded into (X+Y).
  R3  The qsGW matrix of Eq. (Sigma.c.qsGW.real) takes the real part of
      Eq. (Sigma.c.GW): 1/(x -/+ i eta) -> x/(x^2 + eta^2).
  R4  (P|mu nu) are RI factors already contracted with the Coulomb metric.
  R5  H0 = h + J with h_MO = diag(eps0) - J0 - Sigma_x0 (input read as an HF
      solution) unless h is supplied; h_MO follows the orbital rotation.
  R6  Aufbau occupations of the sorted updated energies; no mixing.
  R11 Second-order exchange of Eq. (Sigma.c.MP2) for an occupied summed
      orbital p (the 2h1p part): the factor is (p a|i n), the one the
      antisymmetrised second-order expansion gives; the printed (p i|a n) is that
      expansion's factor only for an empty p (the 2p1h part), which is kept.
  R12 G0W0 (the diagonal m = n of Eq. (Sigma.c.GW)): the quasiparticle
      equation is solved to first order around eps_p (renormalisation factor Z_p),
      starting from the input mean field whose potential is v = diag(eps) - h - J.
  R13 Open shell: reading R1 for every spin pair of the spin-resolved Casida
      problem (A = D + K, B = K), so X + Y = D^(1/2) Z Omega^(-1/2) with no spin
      factor; h spin independent, read per spin from its HF solution when absent.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# Eq. (AO.to.MO) in RI form
# ----------------------------------------------------------------------------
def ri_mo_transform(L: np.ndarray, C: np.ndarray) -> np.ndarray:
    """B^P_pq = sum_{mu nu} C_{mu p} (P|mu nu) C_{nu q}.

    Eq. (AO.to.MO) contracts the four AO indices of (mu nu|la ta) with C; with
    (mu nu|la ta) = sum_P (P|mu nu)(P|la ta) (reading R4) the same contraction
    acts on each three-centre factor, so (pq|rs) = sum_P B^P_pq B^P_rs (Eq. MO.4.ERI).
    L: [na, nb, nb], C: [nb, nb] with column p the MO p (Eq. MO).
    """
    na = L.shape[0]
    B = np.empty_like(L)
    for P in range(na):
        B[P] = C.T @ L[P] @ C
    return B


def transitions(n_basis: int, n_occ: int):
    """(i, a) of each transition t = i*nv + (a - no), occupied-major."""
    nv = n_basis - n_occ
    i = np.repeat(np.arange(n_occ), nv)
    a = np.tile(np.arange(n_occ, n_basis), n_occ)
    return i, a


# ----------------------------------------------------------------------------
# Eqs. (Casida.AB.XY), (Casida.A), (Casida.B)
# ----------------------------------------------------------------------------
def casida_AB(B: np.ndarray, eps: np.ndarray, n_occ: int):
    """Singlet (spin-summed) Casida blocks A and B.

    Eq. (Casida.A): A = (eps_a - eps_i) delta + kernel, Eq. (Casida.B): B = kernel,
    with the Coulomb kernel (ia sigma|jb sigma') summed over the two spins of a
    closed shell (factor 2) and the "+" sign of reading R1.
    Returns (A, Bc, D) with D_t = eps_a - eps_i.
    """
    nb = eps.shape[0]
    i, a = transitions(nb, n_occ)
    D = eps[a] - eps[i]
    Bia = B[:, i, a]                 # [na, n_ov]: B^P_{ia}
    K = Bia.T @ Bia                  # K_tu = (ia|jb) = sum_P B^P_ia B^P_jb
    A = np.diag(D) + 2.0 * K
    Bc = 2.0 * K
    return A, Bc, D


def casida_M(A: np.ndarray, Bc: np.ndarray, D: np.ndarray) -> np.ndarray:
    """Symmetric reduction of Eq. (Casida.AB.XY) for real orbitals.

    (A - B)^(1/2) (A + B) (A - B)^(1/2) Z = Omega^2 Z.  Here A - B = diag(D),
    so M = D^(1/2) (A + B) D^(1/2) = D^2 + 4 D^(1/2) K D^(1/2).
    """
    sq = np.sqrt(D)
    return sq[:, None] * (A + Bc) * sq[None, :]


def casida_M_apply(B: np.ndarray, eps: np.ndarray, n_occ: int):
    """The product x -> M x of the symmetric reduction of Eq. (Casida.AB.XY) without
    forming M: M x = D^2 x + 4 D^(1/2) B_ia^T (B_ia (D^(1/2) x)), with K = B_ia^T B_ia of
    Eq. (Casida.A/B) applied as two products over the auxiliary index (for workloads
    whose n_ov x n_ov matrix is too large to form on the host).  Returns (apply, D)."""
    nb = eps.shape[0]
    i, a = transitions(nb, n_occ)
    D = eps[a] - eps[i]
    Bia = np.ascontiguousarray(B[:, i, a])        # [na, n_ov]
    sq = np.sqrt(D)

    def apply(x):
        x = np.asarray(x, dtype=np.float64)
        y = sq[:, None] * x if x.ndim == 2 else sq * x
        k = Bia.T @ (Bia @ y)
        return (D * D)[:, None] * x + 4.0 * (sq[:, None] * k) if x.ndim == 2 else D * D * x + 4.0 * sq * k

    return apply, D


def rpa_eigensolve(M: np.ndarray, D: np.ndarray):
    """Omega_s ascending and (X+Y)^s from the eigenpairs of M.

    With M Z = Z Lambda: Omega = sqrt(Lambda) and, normalising (X-Y)^T (X+Y) = 1,
    X + Y = (A - B)^(1/2) Z Omega^(-1/2).  The closed-shell spin sum of
    Eq. (w.residue) contributes sqrt(2) (reading R2), folded in here:
    (X+Y)_ts = sqrt(2) sqrt(D_t) Z_ts / sqrt(Omega_s).
    Eigenvector gauge: the largest-magnitude component of each Z column is positive.
    """
    lam, Z = np.linalg.eigh(M)
    if lam[0] <= 0.0:
        raise FloatingPointError("RPA instability: M has a non-positive eigenvalue")
    Z = fix_gauge(Z)
    Omega = np.sqrt(lam)
    XpY = np.sqrt(2.0) * np.sqrt(D)[:, None] * Z / np.sqrt(Omega)[None, :]
    return Omega, XpY, Z


def fix_gauge(Z: np.ndarray) -> np.ndarray:
    """Flip each column so that its largest-magnitude entry is positive."""
    idx = np.argmax(np.abs(Z), axis=0)
    s = np.sign(Z[idx, np.arange(Z.shape[1])])
    s[s == 0] = 1.0
    return Z * s[None, :]


# ----------------------------------------------------------------------------
# Eq. (w.residue)
# ----------------------------------------------------------------------------
def gw_residues(B: np.ndarray, XpY: np.ndarray, n_occ: int):
    """w^s_pq = sum_{ia} (pq|ia) (X+Y)^s_ia = sum_P B^P_pq R_Ps, R = B_ia^T-weighted.

    R_Ps = sum_t B^P_t (X+Y)_ts (t = ia); returns (R [na, n_ov], w [n_ov, nb, nb]).
    """
    R = residue_weights(B, XpY, n_occ)
    w = np.einsum("Ppq,Ps->spq", B, R, optimize=True)
    return R, w


def residue_weights(B: np.ndarray, XpY: np.ndarray, n_occ: int) -> np.ndarray:
    """R_Ps = sum_t B^P_t (X+Y)_ts over the transitions t = ia: the auxiliary side of
    Eq. (w.residue), so that w^s_pq = sum_P B^P_pq R_Ps.  [na, n_ov]."""
    nb = B.shape[1]
    i, a = transitions(nb, n_occ)
    return B[:, i, a] @ XpY


def residues_of_state(B: np.ndarray, R: np.ndarray, m: int) -> np.ndarray:
    """w^s_pm for one orbital m, every (p, s): sum_P B^P_pm R_Ps (Eq. w.residue). [p, s]."""
    return B[:, :, m].T @ R


# ----------------------------------------------------------------------------
# Eq. (K): exchange, and Eq. (J): Hartree, in the MO basis
# ----------------------------------------------------------------------------
def sigma_x(B: np.ndarray, n_occ: int) -> np.ndarray:
    """Sigma_x,pq = -sum_i (p i|i q) = -sum_i sum_P B^P_pi B^P_qi (Eq. K, one spin)."""
    Bo = B[:, :, :n_occ]            # [na, nb, no]
    return -np.einsum("Ppi,Pqi->pq", Bo, Bo, optimize=True)


def hartree(B: np.ndarray, n_occ: int) -> np.ndarray:
    """J_pq = sum_{sigma} sum_i (pq|ii) = 2 sum_P B^P_pq sum_i B^P_ii (Eqs. J, D)."""
    rho = np.einsum("Pii->P", B[:, :n_occ, :n_occ])
    return 2.0 * np.einsum("Ppq,P->pq", B, rho, optimize=True)


# ----------------------------------------------------------------------------
# Eqs. (Sigma.c.GW) and (Sigma.c.qsGW.real)
# ----------------------------------------------------------------------------
def g_real(x, eta: float):
    """Re 1/(x -/+ i eta) = x / (x^2 + eta^2) (reading R3; same for both signs)."""
    return x / (x * x + eta * eta)


def sigma_c_rows(w: np.ndarray, eps: np.ndarray, Omega: np.ndarray, n_occ: int,
                 eta: float) -> np.ndarray:
    """S_pq = Re Sigma^GW_c,pq(omega = eps_p), Eq. (Sigma.c.GW).

    Sigma_pq(w) = sum_{i,s} w^s_pi w^s_qi / (w - eps_i + Omega_s - i eta)
                + sum_{a,s} w^s_pa w^s_qa / (w - eps_a - Omega_s + i eta).
    Row p is taken at omega = eps_p.  The sum over the state m (= i or a) is a
    loop; the sum over s for all (p, q) of one m is a matrix product.
    """
    nb = eps.shape[0]
    S = np.zeros((nb, nb))
    for m in range(nb):
        shift = Omega if m < n_occ else -Omega        # -eps_i + Omega_s | -eps_a - Omega_s
        x = eps[:, None] - eps[m] + shift[None, :]    # [p, s]
        wm = w[:, :, m].T                             # [p, s] = w^s_pm
        S += (wm * g_real(x, eta)) @ wm.T
    return S


def sigma_c_rows_from_R(B: np.ndarray, R: np.ndarray, eps: np.ndarray, Omega: np.ndarray,
                        n_occ: int, eta: float) -> np.ndarray:
    """``sigma_c_rows`` with the residues of each orbital m formed inside the loop over
    m (``residues_of_state``), so that w [n_ov, nb, nb] is never held whole (it is
    33 GB at n_basis = 400).  The same sums in the same order as ``sigma_c_rows``."""
    nb = eps.shape[0]
    S = np.zeros((nb, nb))
    for m in range(nb):
        shift = Omega if m < n_occ else -Omega
        x = eps[:, None] - eps[m] + shift[None, :]
        wm = residues_of_state(B, R, m)
        S += (wm * g_real(x, eta)) @ wm.T
    return S


def sigma_c_qs(S: np.ndarray) -> np.ndarray:
    """Eq. (Sigma.c.qsGW.real): 1/2 [Sigma_mn(eps_n) + Sigma_nm(eps_m)] = 1/2 (S + S^T)^T."""
    return 0.5 * (S + S.T)


def sigma_c_at(w: np.ndarray, eps: np.ndarray, Omega: np.ndarray, n_occ: int,
               eta: float, omega: float) -> np.ndarray:
    """Re Sigma^GW_c,pq(omega) for one frequency, all (p, q) (Eq. Sigma.c.GW)."""
    nb = eps.shape[0]
    out = np.zeros((nb, nb))
    for m in range(nb):
        shift = Omega if m < n_occ else -Omega
        gm = g_real(omega - eps[m] + shift, eta)     # [s]
        wm = w[:, :, m]                               # [s, p]
        out += (wm * gm[:, None]).T @ wm
    return out


# ----------------------------------------------------------------------------
# G0W0: the diagonal of Eq. (Sigma.c.GW) at eps_p, linearised (reading R12)
# ----------------------------------------------------------------------------
def g_real_derivative(x, eta: float):
    """d/dx of x / (x^2 + eta^2) = (eta^2 - x^2) / (x^2 + eta^2)^2."""
    d = x * x + eta * eta
    return (eta * eta - x * x) / (d * d)


def sigma_c_diag(w: np.ndarray, eps: np.ndarray, Omega: np.ndarray, n_occ: int, eta: float):
    """Re Sigma^GW_c,pp(omega) and its omega-derivative at omega = eps_p, every p.

    Sigma_pp(w) = sum_{m,s} (w^s_pm)^2 g(w - eps_m +/- Omega_s), Eq. (Sigma.c.GW) with
    m = n, + Omega_s for occupied m and - Omega_s for empty m.
    """
    nb = eps.shape[0]
    sig = np.zeros(nb)
    dsig = np.zeros(nb)
    for m in range(nb):
        shift = Omega if m < n_occ else -Omega
        x = eps[:, None] - eps[m] + shift[None, :]        # [p, s]
        w2 = w[:, :, m].T ** 2                             # [p, s]
        sig += np.sum(w2 * g_real(x, eta), axis=1)
        dsig += np.sum(w2 * g_real_derivative(x, eta), axis=1)
    return sig, dsig


def g0w0_pass(L: np.ndarray, eps: np.ndarray, C: np.ndarray, n_occ: int, eta: float,
              h_mo: np.ndarray | None = None) -> dict:
    """One-shot G0W0 from (eps, C): Eqs. (AO.to.MO) -> (Casida) -> (w.residue) ->
    the diagonal of (Sigma.c.GW), and the linearised quasiparticle equation
      eps^QP_p = eps_p + Z_p [Sigma_x,pp + Sigma_c,pp(eps_p) - v_pp],
      Z_p = 1 / (1 - dSigma_c,pp/dw (eps_p)),  v = diag(eps) - h_MO - J   (reading R12).
    With h derived from the input read as HF (reading R5) Sigma_x,pp - v_pp = 0."""
    B = ri_mo_transform(L, C)
    J = hartree(B, n_occ)
    Sx = sigma_x(B, n_occ)
    if h_mo is None:
        h_mo = hf_core_mo(B, eps, n_occ)
    A, Bc, D = casida_AB(B, eps, n_occ)
    Omega, XpY, _ = rpa_eigensolve(casida_M(A, Bc, D), D)
    _, w = gw_residues(B, XpY, n_occ)
    sig, dsig = sigma_c_diag(w, eps, Omega, n_occ, eta)
    v = eps - np.diag(h_mo) - np.diag(J)
    Z = 1.0 / (1.0 - dsig)
    eqp = eps + Z * (np.diag(Sx) + sig - v)
    return {"Omega": Omega, "w": w, "sigma_c_diag": sig, "dsigma_c_diag": dsig, "Z": Z,
            "eps_qp": eqp, "sigma_x_diag": np.diag(Sx).copy(), "v_diag": v}


# ----------------------------------------------------------------------------
# Eqs. (Sigma.c.MP2) and (Sigma.c.qsMP2.real): the qsMP2 self-energy
# ----------------------------------------------------------------------------
def mp2_factors(B: np.ndarray, n_occ: int, p: int):
    """The two integral factors of Eq. (Sigma.c.MP2) for one summed orbital p.

    Returns (Ap, Xp), both [n, t] over all orbitals n and transitions t = (i, a):
      Ap[n, t] = (n p|i a) = sum_P B^P_np B^P_ia           (direct factor),
      Xp[n, t] = (p a|i n) for occupied p, (p i|a n) for empty p  (exchange
      partner, reading R11), each = sum_P B^P_.. B^P_.. (Eq. MO.4.ERI).
    Each factor is one matrix product over P.
    """
    na, nb = B.shape[0], B.shape[1]
    nv = nb - n_occ
    i, a = transitions(nb, n_occ)
    Ap = B[:, :, p].T @ B[:, i, a]                                       # [n, t]
    if p < n_occ:
        # (p a|i n) = sum_P B^P_pa B^P_in: [a, (i, n)] -> [n, (i, a)]
        X = B[:, p, n_occ:].T @ B[:, :n_occ, :].reshape(na, n_occ * nb)
        Xp = X.reshape(nv, n_occ, nb).transpose(2, 1, 0)
    else:
        # (p i|a n) = sum_P B^P_pi B^P_an: [i, (a, n)] -> [n, (i, a)]
        X = B[:, p, :n_occ].T @ B[:, n_occ:, :].reshape(na, nv * nb)
        Xp = X.reshape(n_occ, nv, nb).transpose(2, 0, 1)
    return Ap, Xp.reshape(nb, n_occ * nv)


def sigma_mp2_at(B: np.ndarray, eps: np.ndarray, n_occ: int, eta: float,
                 omega: float) -> np.ndarray:
    """Re Sigma^MP2_c,mn(omega) for one frequency, all (m, n) (Eq. Sigma.c.MP2).

    Sigma_mn(w) = sum_{p,i,a} (m p|i a) [2 (p n|a i) - X_p(n; i, a)] h_p(w; i, a),
    the factor 2 being the closed-shell sum over sigma' of the direct term and
    h_p = Re 1/(w + e_a - e_i - e_p - i eta) for occupied p,
          Re 1/(w + e_i - e_a - e_p + i eta) for empty p   (reading R3).
    """
    nb = eps.shape[0]
    i, a = transitions(nb, n_occ)
    D = eps[a] - eps[i]
    out = np.zeros((nb, nb))
    for p in range(nb):
        Ap, Xp = mp2_factors(B, n_occ, p)
        x = omega - eps[p] + (D if p < n_occ else -D)
        out += (Ap * g_real(x, eta)[None, :]) @ (2.0 * Ap - Xp).T
    return out


def sigma_mp2_rows(B: np.ndarray, eps: np.ndarray, n_occ: int, eta: float) -> np.ndarray:
    """S_mn = Re Sigma^MP2_c,mn(omega = eps_m), Eq. (Sigma.c.MP2): row m at its own energy.

    The same sum as ``sigma_mp2_at`` with the denominator taken per row.  The
    qsMP2 matrix of Eq. (Sigma.c.qsMP2.real) is then 1/2 (S + S^T)
    (``sigma_c_qs``), since Sigma^MP2(w) is symmetric for real orbitals.
    """
    nb = eps.shape[0]
    i, a = transitions(nb, n_occ)
    D = eps[a] - eps[i]
    S = np.zeros((nb, nb))
    for p in range(nb):
        Ap, Xp = mp2_factors(B, n_occ, p)
        x = eps[:, None] - eps[p] + (D if p < n_occ else -D)[None, :]   # [m, t]
        S += (Ap * g_real(x, eta)) @ (2.0 * Ap - Xp).T
    return S


# ----------------------------------------------------------------------------
# Eqs. (H), (GEP): quasiparticle update
# ----------------------------------------------------------------------------
def hf_core_mo(B: np.ndarray, eps: np.ndarray, n_occ: int) -> np.ndarray:
    """h_MO = diag(eps) - J - Sigma_x: the one-body part that makes (eps, C) an
    HF solution of Eq. (H) with Sigma_c = 0 (reading R5)."""
    return np.diag(eps) - hartree(B, n_occ) - sigma_x(B, n_occ)


def qs_update(h_mo: np.ndarray, J: np.ndarray, Sx: np.ndarray, Sc: np.ndarray,
              C: np.ndarray):
    """Solve H U = U diag(eps') with H = h + J + Sigma_x + Sigma_c (Eqs. H, GEP, S = I).

    Returns (eps' ascending, C' = C U, h_MO' = U^T h_MO U, U), gauge as fix_gauge.
    """
    H = h_mo + J + Sx + Sc
    H = 0.5 * (H + H.T)
    e, U = np.linalg.eigh(H)
    U = fix_gauge(U)
    return e, C @ U, U.T @ h_mo @ U, U


# ----------------------------------------------------------------------------
# One qsGW iteration
# ----------------------------------------------------------------------------
def qsgw_pass(L: np.ndarray, eps: np.ndarray, C: np.ndarray, n_occ: int,
              eta: float, h_mo: np.ndarray | None = None, correlation: bool = True,
              keep_w: bool = True) -> dict:
    """One RI-qsGW iteration: Eqs. (AO.to.MO) -> (Casida) -> (w.residue) ->
    (Sigma.c.GW, Sigma.c.qsGW.real, K) -> (H, GEP).

    ``h_mo`` is the one-body Hamiltonian in the basis of the current orbitals; if
    None it is derived from the input read as an HF solution (reading R5).
    ``correlation=False`` sets Sigma_c = 0 (the exchange-only limit).
    ``keep_w=False`` forms the residues of one orbital m at a time inside the sum
    of Eq. (Sigma.c.GW) and returns w = None (for workloads whose w does not fit
    in host memory); the values are the same.
    Returns every intermediate and the updated (eps', C', h_MO').
    """
    B = ri_mo_transform(L, C)
    if h_mo is None:
        h_mo = hf_core_mo(B, eps, n_occ)
    A, Bc, D = casida_AB(B, eps, n_occ)
    M = casida_M(A, Bc, D)
    del A, Bc
    Omega, XpY, Z = rpa_eigensolve(M, D)
    if keep_w:
        R, w = gw_residues(B, XpY, n_occ)
    else:
        R, w = residue_weights(B, XpY, n_occ), None
    Sx = sigma_x(B, n_occ)
    if correlation and keep_w:
        Sc = sigma_c_qs(sigma_c_rows(w, eps, Omega, n_occ, eta))
    elif correlation:
        Sc = sigma_c_qs(sigma_c_rows_from_R(B, R, eps, Omega, n_occ, eta))
    else:
        Sc = np.zeros_like(Sx)
    J = hartree(B, n_occ)
    eps_new, C_new, h_new, U = qs_update(h_mo, J, Sx, Sc, C)
    return {
        "B": B, "D": D, "M": M, "Omega": Omega, "XpY": XpY, "Z": Z, "R": R, "w": w,
        "sigma_x": Sx, "sigma_c": Sc, "J": J, "h_mo": h_mo,
        "eps_new": eps_new, "C_new": C_new, "h_mo_new": h_new, "U": U,
    }


def qsmp2_pass(L: np.ndarray, eps: np.ndarray, C: np.ndarray, n_occ: int,
               eta: float, h_mo: np.ndarray | None = None) -> dict:
    """One RI-qsMP2 iteration: Eqs. (AO.to.MO) -> (Sigma.c.MP2, Sigma.c.qsMP2.real, K)
    -> (H, GEP).  No RPA: the correlation self-energy is second order in v."""
    B = ri_mo_transform(L, C)
    if h_mo is None:
        h_mo = hf_core_mo(B, eps, n_occ)
    Sx = sigma_x(B, n_occ)
    Sc = sigma_c_qs(sigma_mp2_rows(B, eps, n_occ, eta))
    J = hartree(B, n_occ)
    eps_new, C_new, h_new, U = qs_update(h_mo, J, Sx, Sc, C)
    return {"B": B, "sigma_x": Sx, "sigma_c": Sc, "J": J, "h_mo": h_mo,
            "eps_new": eps_new, "C_new": C_new, "h_mo_new": h_new, "U": U}


def qsmp2_iterations(L, eps, C, n_occ, eta, n_iter, h_mo=None) -> list:
    """n_iter successive qsMP2 iterations, each starting from the previous (eps', C')."""
    out = []
    for _ in range(n_iter):
        r = qsmp2_pass(L, eps, C, n_occ, eta, h_mo)
        out.append(r)
        eps, C, h_mo = r["eps_new"], r["C_new"], r["h_mo_new"]
    return out


# ----------------------------------------------------------------------------
# Open shell: the sigma-resolved equations of Sec. II (GEP, H, J, D, K,
# Casida.AB.XY, Casida.A/B, w.residue, Sigma.c.GW) with one set of orbitals per spin
# ----------------------------------------------------------------------------
def casida_M_open(Bs, epss, n_occs):
    """M = D^(1/2) (A + B) D^(1/2) over the transitions of both spins, up first.

    Eqs. (Casida.A/B) with spins written out: A_{t s, u s'} = D_t delta + (t s|u s'),
    B_{t s, u s'} = (t s|u s') ("+" sign, reading R1), so A - B = diag(D) and
    M = D^2 + 2 D^(1/2) K D^(1/2) with K_{t s, u s'} = sum_P B^{P s}_t B^{P s'}_u.
    Returns (M, D, Bt [na, n_ov_up + n_ov_dn]).
    """
    Dl, Bl = [], []
    for B, eps, no in zip(Bs, epss, n_occs):
        i, a = transitions(eps.shape[0], no)
        Dl.append(eps[a] - eps[i])
        Bl.append(B[:, i, a])
    D = np.concatenate(Dl)
    Bt = np.concatenate(Bl, axis=1)
    K = Bt.T @ Bt
    sq = np.sqrt(D)
    return np.diag(D * D) + 2.0 * sq[:, None] * K * sq[None, :], D, Bt


def rpa_eigensolve_open(M: np.ndarray, D: np.ndarray):
    """Omega ascending and X + Y = D^(1/2) Z Omega^(-1/2) (no spin factor: the sum over
    sigma' of Eq. (w.residue) runs over the spin-resolved transitions themselves)."""
    lam, Z = np.linalg.eigh(M)
    if lam[0] <= 0.0:
        raise FloatingPointError("RPA instability: M has a non-positive eigenvalue")
    Z = fix_gauge(Z)
    Omega = np.sqrt(lam)
    return Omega, np.sqrt(D)[:, None] * Z / np.sqrt(Omega)[None, :], Z


def hartree_open(B: np.ndarray, Bs, n_occs) -> np.ndarray:
    """J_pq in the basis of B's orbitals: sum_P B^P_pq sum_{s} sum_{i in occ s} B^{P s}_ii (Eq. J)."""
    rho = sum(np.einsum("Pii->P", Bx[:, :no, :no]) for Bx, no in zip(Bs, n_occs))
    return np.einsum("Ppq,P->pq", B, rho, optimize=True)


def qsgw_pass_open(L, epss, Cs, n_occs, eta, h_mos=None) -> dict:
    """One open-shell RI-qsGW iteration; epss, Cs, n_occs, h_mos are (up, down) pairs.

    Per spin s: B^s = C^sT L C^s; the spin-resolved Casida problem (casida_M_open);
    w^{v}_{pq s} = sum_P B^{P s}_pq R_Pv with R = Bt (X+Y); Sigma_c^s from Eq.
    (Sigma.c.GW) with the spin-s energies and occupations, made static by Eq.
    (Sigma.c.qsGW.real); Sigma_x^s = -sum_{i in occ s} (p i s|i q s); J from both
    spins; H^s = h^s + J^s + Sigma_x^s + Sigma_c^s (Eqs. H, GEP).  h^s defaults to
    the HF reading R5 applied per spin.
    """
    Bs = [ri_mo_transform(L, C) for C in Cs]
    M, D, Bt = casida_M_open(Bs, epss, n_occs)
    Omega, XpY, Z = rpa_eigensolve_open(M, D)
    R = Bt @ XpY
    out = {"Omega": Omega, "D": D, "M": M, "XpY": XpY, "R": R, "spin": []}
    for k, (B, eps, C, no) in enumerate(zip(Bs, epss, Cs, n_occs)):
        w = np.einsum("Ppq,Ps->spq", B, R, optimize=True)
        Sx = sigma_x(B, no)
        J = hartree_open(B, Bs, n_occs)
        h = h_mos[k] if h_mos is not None else np.diag(eps) - J - Sx
        Sc = sigma_c_qs(sigma_c_rows(w, eps, Omega, no, eta))
        eps_new, C_new, h_new, U = qs_update(h, J, Sx, Sc, C)
        out["spin"].append({"B": B, "w": w, "sigma_x": Sx, "sigma_c": Sc, "J": J, "h_mo": h,
                            "eps_new": eps_new, "C_new": C_new, "h_mo_new": h_new})
    return out


def qsgw_iterations(L, eps, C, n_occ, eta, n_iter, h_mo=None) -> list:
    """n_iter successive qsGW iterations, each starting from the previous (eps', C')."""
    out = []
    for _ in range(n_iter):
        r = qsgw_pass(L, eps, C, n_occ, eta, h_mo)
        out.append(r)
        eps, C, h_mo = r["eps_new"], r["C_new"], r["h_mo_new"]
    return out
