"""Brute-force forms of the same equations, for tiny inputs only.

TEST INFRASTRUCTURE ONLY (same import rule as ``oracle.qsgw``).  These functions
take the paper's equations with every index written out -- explicit spins,
four-index integrals, nested loops, a project-written Jacobi eigensolver -- so
that the matrix forms in ``oracle.qsgw`` can be checked against them.
"""
from __future__ import annotations

import math

import numpy as np


def eri_ao(L: np.ndarray) -> np.ndarray:
    """(mu nu|la ta) = sum_P (P|mu nu)(P|la ta) (Eq. AO.4.ERI under the RI reading)."""
    return np.einsum("Pmn,Plt->mnlt", L, L)


def eri_mo(L: np.ndarray, C: np.ndarray) -> np.ndarray:
    """(pq|rs) by the four-index AO->MO transformation of Eq. (AO.to.MO), one index at a time."""
    g = eri_ao(L)
    g = np.einsum("mp,mnlt->pnlt", C, g)
    g = np.einsum("nq,pnlt->pqlt", C, g)
    g = np.einsum("lr,pqlt->pqrt", C, g)
    return np.einsum("ts,pqrt->pqrs", C, g)


def density_ao(C: np.ndarray, n_occ: int) -> np.ndarray:
    """Eq. (D) for one spin: D_mu nu = sum_m f_m C_mu m C_nu m, f = 1 for the lowest n_occ."""
    Co = C[:, :n_occ]
    return Co @ Co.T


def hartree_exchange_mo(L: np.ndarray, C: np.ndarray, n_occ: int):
    """J (Eq. J, both spins) and -K (Eq. K, one spin) in the AO basis, then in the MO basis."""
    g = eri_ao(L)
    D = density_ao(C, n_occ)
    J = np.einsum("mnlt,lt->mn", g, 2.0 * D)
    K = np.einsum("lt,mltn->mn", D, g)
    return C.T @ J @ C, -(C.T @ K @ C)


def casida_spin_orbital(L: np.ndarray, C: np.ndarray, eps: np.ndarray, n_occ: int):
    """Full non-Hermitian Casida problem of Eq. (Casida.AB.XY) over spin orbitals.

    Rows/columns run over (i, a, sigma), sigma in {up, down}, i-major then a then sigma.
    A = (eps_a - eps_i) delta delta delta_{sigma sigma'} + (ia sigma|jb sigma'),
    B = (ia sigma|bj sigma'), with the "+" Coulomb sign (reading R1).  For real
    orbitals the integral is independent of the spins.
    Returns (eigenvalues ascending, right eigenvectors (X;Y) as columns, ERIs).
    """
    nb = eps.shape[0]
    g = eri_mo(L, C)
    occ = range(n_occ)
    vir = range(n_occ, nb)
    idx = [(i, a, s) for i in occ for a in vir for s in (0, 1)]
    n = len(idx)
    A = np.zeros((n, n))
    Bm = np.zeros((n, n))
    for u, (i, a, s) in enumerate(idx):
        for v, (j, b, sp) in enumerate(idx):
            A[u, v] = g[i, a, j, b] + ((eps[a] - eps[i]) if (i == j and a == b and s == sp) else 0.0)
            Bm[u, v] = g[i, a, b, j]
    big = np.block([[A, Bm], [-Bm, -A]])
    vals, vecs = np.linalg.eig(big)
    order = np.argsort(vals.real)
    return vals.real[order], vecs.real[:, order], g, idx


def singlet_residues_spin_orbital(L, C, eps, n_occ, tol=1e-8):
    """Positive Casida frequencies with non-zero residue and w^s_mn of Eq. (w.residue).

    w^s_mn = sum_{i a sigma'} (mn|ia sigma') (X^s + Y^s)_{ia sigma'}, with (X, Y)
    normalised by X^T X - Y^T Y = 1.  Spin-flip (triplet) combinations have zero
    residue and are returned separately.
    Returns (Omega_singlet, w [n_s, nb, nb], Omega_triplet).
    """
    vals, vecs, g, idx = casida_spin_orbital(L, C, eps, n_occ)
    n = len(idx)
    nb = eps.shape[0]
    sing_O, sing_w, trip_O = [], [], []
    for k in range(2 * n):
        if vals[k] <= 0:
            continue
        X, Y = vecs[:n, k], vecs[n:, k]
        norm = X @ X - Y @ Y
        X, Y = X / math.sqrt(norm), Y / math.sqrt(norm)
        w = np.zeros((nb, nb))
        for u, (i, a, s) in enumerate(idx):
            w += g[:, :, i, a] * (X[u] + Y[u])
        if np.max(np.abs(w)) > tol:
            sing_O.append(vals[k])
            sing_w.append(w)
        else:
            trip_O.append(vals[k])
    return np.array(sing_O), np.array(sing_w), np.array(trip_O)


def casida_spin_orbital_open(L: np.ndarray, Cs, epss, n_occs):
    """Full non-Hermitian Casida problem of Eq. (Casida.AB.XY) over spin orbitals with
    one set of MOs per spin: rows/columns (i, a, s), spin up first.

    A = (e_a^s - e_i^s) delta + (i a s|j b s'), B = (i a s|b j s'), the integrals
    (pq s|rt s') = sum C^s C^s C^s' C^s' (mu nu|la ta) by the four-index transformation
    of Eq. (AO.to.MO) with the "+" Coulomb sign (reading R1).
    Returns eigenvalues ascending.
    """
    g = eri_ao(L)
    gmo = {}
    for s1 in (0, 1):
        for s2 in (0, 1):
            x = np.einsum("mp,mnlt->pnlt", Cs[s1], g)
            x = np.einsum("nq,pnlt->pqlt", Cs[s1], x)
            x = np.einsum("lr,pqlt->pqrt", Cs[s2], x)
            gmo[s1, s2] = np.einsum("ts,pqrt->pqrs", Cs[s2], x)
    nb = Cs[0].shape[0]
    idx = [(i, a, s) for s in (0, 1) for i in range(n_occs[s]) for a in range(n_occs[s], nb)]
    n = len(idx)
    A = np.zeros((n, n))
    Bm = np.zeros((n, n))
    for u, (i, a, s) in enumerate(idx):
        for v, (j, b, sp) in enumerate(idx):
            A[u, v] = gmo[s, sp][i, a, j, b] + ((epss[s][a] - epss[s][i]) if u == v else 0.0)
            Bm[u, v] = gmo[s, sp][i, a, b, j]
    vals = np.linalg.eigvals(np.block([[A, Bm], [-Bm, -A]]))
    return np.sort(vals.real)


def sigma_c_loops(w, eps, Omega, n_occ, eta, omega_rows=True):
    """Re Sigma_c,pq(eps_p) by four nested loops over p, q, m, s (Eq. Sigma.c.GW)."""
    nb = eps.shape[0]
    ns = Omega.shape[0]
    S = np.zeros((nb, nb))
    for p in range(nb):
        om = eps[p]
        for q in range(nb):
            acc = 0.0
            for m in range(nb):
                for s in range(ns):
                    if m < n_occ:
                        x = om - eps[m] + Omega[s]
                    else:
                        x = om - eps[m] - Omega[s]
                    acc += w[s, p, m] * w[s, q, m] * x / (x * x + eta * eta)
            S[p, q] = acc
    return S


def sigma_mp2_direct(g: np.ndarray, eps: np.ndarray, n_occ: int, eta: float, omega: float):
    """Re of the direct (first) term of Eq. (Sigma.c.MP2) at one frequency, all (m, n).

    sum_{i a p sigma'} (mp|ia)(pn|ai) [f_p / (w + e_a - e_i - e_p - i eta)
                                     + (1 - f_p) / (w + e_i - e_a - e_p + i eta)],
    with the sigma' sum giving a factor 2 for a closed shell.
    """
    nb = eps.shape[0]
    out = np.zeros((nb, nb))
    for p in range(nb):
        fp = 1.0 if p < n_occ else 0.0
        for i in range(n_occ):
            for a in range(n_occ, nb):
                if fp:
                    x = omega + eps[a] - eps[i] - eps[p]
                else:
                    x = omega + eps[i] - eps[a] - eps[p]
                gx = x / (x * x + eta * eta)
                out += 2.0 * np.outer(g[:, p, i, a], g[p, :, a, i]) * gx
    return out


def antisymmetrised_spin_orbital(g: np.ndarray) -> np.ndarray:
    """<PQ||RS> over spin orbitals P = 2 p + spin, from chemists' (pq|rs) of real orbitals.

    <PQ|RS> = (pr|qs) delta(spin P, spin R) delta(spin Q, spin S); <PQ||RS> = <PQ|RS> - <PQ|SR>.
    """
    nb = g.shape[0]
    n2 = 2 * nb
    sp = np.arange(n2) % 2
    orb = np.arange(n2) // 2
    phys = g[orb[:, None, None, None], orb[None, None, :, None],
             orb[None, :, None, None], orb[None, None, None, :]]          # (p r|q s) at [P, Q, R, S]
    phys = phys * ((sp[:, None, None, None] == sp[None, None, :, None])
                   & (sp[None, :, None, None] == sp[None, None, None, :]))
    return phys - phys.transpose(0, 1, 3, 2)


def sigma2_spin_orbital(g: np.ndarray, eps: np.ndarray, n_occ: int, eta: float, omega: float,
                        part: str = "both") -> np.ndarray:
    """Re of the second-order self-energy over spin orbitals, spatial (m, n) of spin up.

    The antisymmetrised expansion of the self-energy to second order in v:
      Sigma_mn(w) = 1/2 sum_{I A B} <mI||AB><AB||nI> / (w + e_I - e_A - e_B)     (2p1h)
                  + 1/2 sum_{I J A} <mA||IJ><IJ||nA> / (w + e_A - e_I - e_J)     (2h1p)
    with I, J occupied and A, B empty spin orbitals, every sum written out.
    ``part`` selects "2p1h", "2h1p" or "both".
    """
    nb = eps.shape[0]
    asy = antisymmetrised_spin_orbital(g)
    e2 = np.repeat(eps, 2)
    occ = [P for P in range(2 * nb) if P // 2 < n_occ]
    vir = [P for P in range(2 * nb) if P // 2 >= n_occ]
    out = np.zeros((nb, nb))
    for m in range(nb):
        for n in range(nb):
            M, N = 2 * m, 2 * n
            acc = 0.0
            if part in ("both", "2p1h"):
                for I in occ:
                    for A in vir:
                        for Bb in vir:
                            x = omega + e2[I] - e2[A] - e2[Bb]
                            acc += 0.5 * asy[M, I, A, Bb] * asy[A, Bb, N, I] * x / (x * x + eta * eta)
            if part in ("both", "2h1p"):
                for I in occ:
                    for J in occ:
                        for A in vir:
                            x = omega + e2[A] - e2[I] - e2[J]
                            acc += 0.5 * asy[M, A, I, J] * asy[I, J, N, A] * x / (x * x + eta * eta)
            out[m, n] = acc
    return out


def sigma_mp2_printed(g: np.ndarray, eps: np.ndarray, n_occ: int, eta: float, omega: float,
                      part: str = "both") -> np.ndarray:
    """Re of Eq. (Sigma.c.MP2) exactly as printed, four nested loops, one frequency.

    sum_{i a p} [2 (mp|ia)(pn|ai) - (mp|ia)(pi|an)] h_p, with
    h_p = Re 1/(w + e_a - e_i - e_p) for occupied p ("2h1p"), Re 1/(w + e_i - e_a - e_p)
    for empty p ("2p1h").
    """
    nb = eps.shape[0]
    out = np.zeros((nb, nb))
    for p in range(nb):
        occ_p = p < n_occ
        if (part == "2h1p" and not occ_p) or (part == "2p1h" and occ_p):
            continue
        for i in range(n_occ):
            for a in range(n_occ, nb):
                x = omega + (eps[a] - eps[i] - eps[p] if occ_p else eps[i] - eps[a] - eps[p])
                gx = x / (x * x + eta * eta)
                out += np.outer(g[:, p, i, a], 2.0 * g[p, :, a, i] - g[p, i, a, :]) * gx
    return out


def jacobi_eigh(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 100):
    """Cyclic Jacobi eigensolver for a small real symmetric matrix.

    Each rotation zeroes A_pq with the classical angle choice
    (theta = (A_qq - A_pp) / (2 A_pq), t = sign(theta) / (|theta| + sqrt(theta^2 + 1)),
    which is 1 / (2 theta) to working precision once theta^2 would overflow).
    Returns eigenvalues ascending and eigenvectors as columns.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    for _ in range(max_sweeps):
        off = math.sqrt(np.sum((A - np.diag(np.diag(A))) ** 2))
        if off <= tol * max(1.0, math.sqrt(np.sum(A * A))):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                theta = (A[q, q] - A[p, p]) / (2.0 * apq)
                if abs(theta) > 1e150:
                    t = 0.5 / theta
                else:
                    t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                Ap, Aq = A[:, p].copy(), A[:, q].copy()
                A[:, p] = c * Ap - s * Aq
                A[:, q] = s * Ap + c * Aq
                Ap, Aq = A[p, :].copy(), A[q, :].copy()
                A[p, :] = c * Ap - s * Aq
                A[q, :] = s * Ap + c * Aq
                Vp, Vq = V[:, p].copy(), V[:, q].copy()
                V[:, p] = c * Vp - s * Vq
                V[:, q] = s * Vp + c * Vq
    d = np.diag(A).copy()
    order = np.argsort(d)
    return d[order], V[:, order]
