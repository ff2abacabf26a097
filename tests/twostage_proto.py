"""Prototype of the two-stage tridiagonalisation (test-side, not part of the library).

Stage 1, dense -> lower band of width b: for each panel of b columns, the Householder QR of
the part below the band (reflectors H_c = I - tau_c v_c v_c^T, gathered as Q = I - V T V^T,
the compact-WY form), then one two-sided update of the trailing matrix,
    A22 <- Q^T A22 Q = A22 - V Z^T - Z V^T,  Z = A22 V T - 1/2 V (T^T V^T A22 V T),
a symmetric product and a rank-2b update: level-3 work only (the one-stage reduction does half
of its flops as matrix-vector products).

Stage 2, band -> tridiagonal by bulge chasing: sweep j annihilates column j below the
subdiagonal with one reflector on rows j+1..j+b; the similarity fills the next block down,
whose first column is annihilated by the next reflector (rows b further down), and so on off
the end of the matrix.  One reflector of length <= b per block; ~n^2/(2b) reflectors in all,
~12 b^2 flops each on the band (~6 n^2 b flops), in chains that the next sweep can follow a few
blocks behind.

`cost_model` gives both stages' flops and the length of the bulge-chasing critical path.
"""
from __future__ import annotations

import numpy as np


def house(x):
    """v (v[0] = 1), tau, beta with (I - tau v v^T) x = beta e_0 (dlarfg convention)."""
    alpha = float(x[0])
    s = float(np.dot(x[1:], x[1:]))
    v = np.zeros_like(x)
    v[0] = 1.0
    if s == 0.0:
        return v, 0.0, alpha
    beta = -np.copysign(np.sqrt(alpha * alpha + s), alpha)
    v[1:] = x[1:] / (alpha - beta)
    return v, (beta - alpha) / beta, beta


def apply_sym(A, s, e, v, tau):
    """A <- H A H with H = I - tau v v^T acting on indices s..e (dense storage)."""
    if tau == 0.0:
        return
    blk = A[s:e + 1, :]
    A[s:e + 1, :] = blk - tau * np.outer(v, v @ blk)
    blk = A[:, s:e + 1]
    A[:, s:e + 1] = blk - tau * np.outer(blk @ v, v)


def band_reduce(A, b):
    """Stage 1: the lower band of width b of Q^T A Q, by panels of b columns."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    for k in range(0, n - b - 1, b):
        r0 = k + b                                  # first row below the band
        m = n - r0
        nr = min(b, m - 1)                          # reflectors: columns with 2+ rows left
        panel = A[r0:, k:k + b].copy()              # the panel's b columns (k + b <= r0 <= n - 1)
        V = np.zeros((m, nr))
        taus = np.zeros(nr)
        for c in range(nr):                         # QR of the panel, column by column
            v, tau, beta = house(panel[c:, c])
            V[c:, c] = v
            taus[c] = tau
            panel[c:, c:] -= tau * np.outer(v, v @ panel[c:, c:])
        T = np.zeros((nr, nr))                      # compact WY: Q = I - V T V^T
        for c in range(nr):
            T[:c, c] = -taus[c] * (T[:c, :c] @ (V[:, :c].T @ V[:, c]))
            T[c, c] = taus[c]
        A[r0:, k:k + b] = panel
        A[k:k + b, r0:] = panel.T
        A22 = A[r0:, r0:]
        Y = A22 @ V @ T                              # the symmetric product
        Z = Y - 0.5 * V @ (T.T @ (V.T @ Y))
        A[r0:, r0:] = A22 - V @ Z.T - Z @ V.T        # the rank-2b update
    return A


def bulge_chase(A, b):
    """Stage 2: band of width b -> tridiagonal; also returns the reflector count."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    count = 0
    for j in range(n - 2):
        st, ed = j + 1, min(j + b, n - 1)
        if ed - st >= 1:
            v, tau, _ = house(A[st:ed + 1, j])
            apply_sym(A, st, ed, v, tau)
            count += 1
        while True:
            st2, ed2 = ed + 1, min(ed + b, n - 1)
            if ed2 - st2 < 1:
                break
            v, tau, _ = house(A[st2:ed2 + 1, st])  # the bulge's first column
            apply_sym(A, st2, ed2, v, tau)
            count += 1
            st, ed = st2, ed2
    return A, count


def reflector_count(n, b):
    """Reflectors of `bulge_chase` on an n x n band of width b, counted as its loops run."""
    total = 0
    for j in range(n - 2):
        st, ed = j + 1, min(j + b, n - 1)
        total += ed - st >= 1
        while min(ed + b, n - 1) - (ed + 1) >= 1:
            ed = min(ed + b, n - 1)
            total += 1
    return total


def cost_model(n, b=64):
    """Flops of the two stages and the bulge chase's dependent steps (sweeps overlap with a
    lag of ~3 blocks, so about 3 steps per sweep plus one sweep's length)."""
    stage1 = 4.0 / 3.0 * n ** 3
    stage2 = 6.0 * n * n * b
    chain = 3 * n + n // b
    return {"stage1_flops": stage1, "stage2_flops": stage2, "chase_steps": chain,
            "reflectors": n * n / (2.0 * b)}
