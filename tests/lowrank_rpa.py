"""Prototype of the low-rank route to the RPA poles (test-side, not part of the library).

M = D^2 + V V^T with V = 2 D^(1/2) B_ia^T (n_ov x n_aux): a diagonal plus a matrix of
rank n_aux (Eqs. Casida.AB.XY, Casida.A/B with reading R1).  This module restates the
secular (Weinstein-Aronszajn) route that avoids the dense n_ov^3 reduction:

* counting: for lam not in {D_t^2}, the number of eigenvalues of M below lam is
  #{t : D_t^2 < lam} - #{negative eigenvalues of G(lam)},
  G(lam) = I + V^T (D^2 - lam)^(-1) V  (n_aux x n_aux),
  which follows from Haynsworth's inertia additivity applied to the block matrix
  [[D^2 - lam, V], [V^T, -I]] (its two Schur complements are M - lam and -G(lam));
* each eigenvalue by bisection on that count;
* the residue weights without the n_ov-vectors: G(lam_s) y_s = 0 with y_s = V^T z_s
  and z_s = -(D^2 - lam_s)^(-1) V y_s, so R_Ps = sum_t B^P_t (X+Y)_ts =
  y_s,P / (sqrt(2) sqrt(Omega_s)) once z_s has unit norm.

One count costs n_aux^2 n_ov + n_aux^3 flops; all n_ov eigenvalues need ~50 counts
each, i.e. ~50 n_aux^2 n_ov^2 flops against ~(4/3 + 4 n_aux / n_ov) n_ov^3 for the dense
route.  ``cost_model`` gives both; ``time_count`` measures one count.
"""
from __future__ import annotations

import time

import numpy as np


def low_rank_factors(B: np.ndarray, eps: np.ndarray, n_occ: int):
    """D_t = eps_a - eps_i and V = 2 D^(1/2) B_ia^T (t = i nv + (a - no))."""
    nb = eps.shape[0]
    nv = nb - n_occ
    i = np.repeat(np.arange(n_occ), nv)
    a = np.tile(np.arange(n_occ, nb), n_occ)
    D = eps[a] - eps[i]
    V = 2.0 * np.sqrt(D)[:, None] * B[:, i, a].T
    return D, V


def count_below(lam: float, D2: np.ndarray, V: np.ndarray) -> int:
    """Number of eigenvalues of D2 + V V^T below lam (lam not equal to any D2_t)."""
    G = np.eye(V.shape[1]) + V.T @ (V / (D2 - lam)[:, None])
    neg = int(np.sum(np.linalg.eigvalsh(0.5 * (G + G.T)) < 0.0))
    return int(np.sum(D2 < lam)) - neg


def secular_eigvals(D2: np.ndarray, V: np.ndarray, rel_tol: float = 1e-14) -> np.ndarray:
    """All eigenvalues of D2 + V V^T by bisection on the inertia count, ascending."""
    n = D2.shape[0]
    lo0 = float(D2.min())                       # M >= D2 in the Loewner order
    hi0 = float(D2.max() + np.sum(V * V))       # D2_max + tr(V V^T) >= lambda_max
    lam = np.empty(n)
    for k in range(n):
        lo, hi = lo0, hi0
        while hi - lo > rel_tol * max(abs(lo), abs(hi)):
            mid = 0.5 * (lo + hi)
            if mid in (lo, hi):
                break
            if np.any(D2 == mid):
                mid = np.nextafter(mid, hi)
            if count_below(mid, D2, V) > k:
                hi = mid
            else:
                lo = mid
        lam[k] = 0.5 * (lo + hi)
    return lam


def secular_residue_weights(lam: np.ndarray, D: np.ndarray, V: np.ndarray) -> np.ndarray:
    """R[:, s] = y_s / (sqrt(2) sqrt(Omega_s)) from the null vector y_s of G(lam_s), with
    z_s = -(D^2 - lam_s)^(-1) V y_s normalised and its largest entry made positive."""
    D2 = D * D
    na = V.shape[1]
    R = np.empty((na, lam.shape[0]))
    for s, l in enumerate(lam):
        G = np.eye(na) + V.T @ (V / (D2 - l)[:, None])
        w, U = np.linalg.eigh(0.5 * (G + G.T))
        y = U[:, np.argmin(np.abs(w))]
        z = -(V @ y) / (D2 - l)
        nz = np.linalg.norm(z)
        z /= nz
        y = y / nz
        if z[np.argmax(np.abs(z))] < 0.0:
            y = -y
        R[:, s] = y / (np.sqrt(2.0) * np.sqrt(np.sqrt(l)))
    return R


def cost_model(n_ov: int, n_aux: int, counts_per_eigenvalue: int = 50) -> dict:
    """Flops of the two routes to all n_ov poles and the residue weights R."""
    secular = counts_per_eigenvalue * n_ov * (2.0 * n_aux * n_aux * n_ov + n_aux ** 3)
    dense = 4.0 / 3.0 * n_ov ** 3 + 4.0 * n_aux * n_ov ** 2     # reduction + thin back-transformation
    return {"secular_flops": secular, "dense_flops": dense, "ratio": secular / dense}


def time_count(n_ov: int, n_aux: int, seed: int = 0, repeat: int = 3) -> float:
    """Seconds of one inertia count at (n_ov, n_aux) on this host (random D, V)."""
    rng = np.random.default_rng(seed)
    D2 = np.sort(rng.uniform(0.1, 25.0, n_ov))
    V = rng.standard_normal((n_ov, n_aux)) * 0.1
    lam = float(np.median(D2)) + 1e-3
    count_below(lam, D2, V)
    t0 = time.perf_counter()
    for _ in range(repeat):
        count_below(lam, D2, V)
    return (time.perf_counter() - t0) / repeat
