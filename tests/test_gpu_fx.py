"""Fixed-point split precision (MOLGW_PREC_BF16X10) on the BF16 tensor cores.

The engine writes each value of a (row, 1024-element K group) as four integer
BF16 slices times one power of two, sums the slice products of each level in
float32 over 256-element chunks (every partial sum an integer below 2^24, so
exact), combines the levels in 64-bit integers and rounds once per group to
float64.  `fx_model` restates that arithmetic on the CPU; the GPU must agree
with it bit for bit, which checks that the tensor cores' float32 accumulation
is exact on such integers.  The qsGW pass with (d)+(e) on this engine must meet
the mixed-path tolerances of the method: QP energies within 1 meV of the float64
oracle and Sigma within 1e-6 relative.
"""
import numpy as np
import pytest

import synthetic as sy
from helpers import lib_context, load_mol, rel_max
from oracle import qsgw

pytestmark = pytest.mark.gpu
ETA = sy.ETA
MEV = 1e-3 / 27.211386245988       # Ha


def fx_split_model(X, ns=4, group=1024, kblock=64):
    """Scales u[row, group] and the ns integer digits of X (rows x K)."""
    rows, K = X.shape
    kp = -(-K // kblock) * kblock
    Xp = np.zeros((rows, kp))
    Xp[:, :K] = X
    ng = -(-kp // group)
    u = np.empty((rows, ng))
    sl = np.zeros((ns, rows, kp))
    for g in range(ng):
        blk = Xp[:, g * group:(g + 1) * group]
        mx = np.abs(blk).max(axis=1)
        _, e = np.frexp(mx)
        e = np.where(mx > 0, e, 0)
        u[:, g] = np.ldexp(1.0, e - 7)
        T = np.rint(blk * (2.0 ** (8 * (ns - 1)) / u[:, g])[:, None]).astype(np.int64)
        for i in range(ns - 1, 0, -1):               # balanced base-256 digits
            d = ((T + 128) & 255) - 128
            sl[i, :, g * group:(g + 1) * group] = d
            T = (T - d) >> 8
        sl[0, :, g * group:(g + 1) * group] = T
    assert np.abs(sl).max() <= 128
    return sl, u, kp


def fx_model(A, B, ns=4, group=1024):
    """The engine's arithmetic: exact level sums per chunk (256 elements with 4
    digits, 128 with 7), levels combined in integers (two words with 7 digits, joined
    into one 64-bit integer at the end of the group), one rounding per group, groups
    summed in order."""
    chunk = 256 if ns == 4 else 128
    sa, ua, kp = fx_split_model(A, ns)
    sb, ub, _ = fx_split_model(B, ns)
    C = np.zeros((A.shape[0], B.shape[0]))
    for g in range(-(-kp // group)):
        Vh = np.zeros(C.shape, dtype=np.int64)
        Vl = np.zeros(C.shape, dtype=np.int64)
        for c0 in range(g * group, min(kp, (g + 1) * group), chunk):
            c1 = min(kp, c0 + chunk)
            L = []
            for lev in range(ns):
                s = sum(sa[a][:, c0:c1] @ sb[lev - a][:, c0:c1].T for a in range(lev + 1))
                assert np.abs(s).max() < 2.0 ** 24
                L.append(s.astype(np.int64))
            Vh += (L[0] << 24) + (L[1] << 16) + (L[2] << 8) + L[3]
            if ns == 7:
                Vl += (L[4] << 16) + (L[5] << 8) + L[6]
        if ns == 7:
            # floor((2^24 Vh + Vl) / 2^10), one rounding to float64, scale 2^-38 u_a u_b
            v = ((Vh << 14) + (Vl >> 10)).astype(np.float64)
            C = C + v * (2.0 ** -38 * ua[:, g][:, None] * ub[:, g][None, :])
        else:
            v = Vh.astype(np.float64)
            C = C + v * (2.0 ** -24 * ua[:, g][:, None] * ub[:, g][None, :])
    return C


@pytest.mark.parametrize("M,N,K", [(64, 48, 100), (200, 130, 2500), (300, 70, 1024)])
def test_fx_gemm_bitwise_model(M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)) * np.exp(-np.arange(K) / 300.0)[None, :]   # decaying along K
    B = rng.standard_normal((N, K)) * 10.0 ** rng.uniform(-3, 3, size=(N, 1))  # rows of mixed scale
    C = np.empty((M, N))
    with lib_context(precision="bf16x10") as ctx:
        ctx.tc_gemm(A, B, C)
    assert np.array_equal(C, fx_model(A, B))
    ref = A @ B.T
    bound = 2.0 ** -30 * K * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :]
    assert np.all(np.abs(C - ref) <= bound)


def test_fx_gemm_largest_level_sums():
    """Values at the slice limits (y = 127.5 -> digits 127, 128 ... or -128 in the
    lower places): level sums of 256-element chunks reach 2^22 .. 2^23 and must
    stay exact."""
    K = 1024
    A = np.full((128, K), 127.5 / 128.0)
    A[1::2] *= -1.0
    B = np.full((64, K), 127.5 / 128.0)
    C = np.empty((128, 64))
    with lib_context(precision="bf16x10") as ctx:
        ctx.tc_gemm(A, B, C)
    assert np.array_equal(C, fx_model(A, B))
    assert np.array_equal(C, A @ B.T)


@pytest.mark.parametrize("M,N,K", [(64, 48, 100), (200, 130, 2500), (257, 33, 1024)])
def test_fx7_gemm_bitwise_model(M, N, K):
    """Seven digits (the engine of MOLGW_FLAG_EIG_TC): bit-exact against the model
    and within float64 accuracy of the exact product."""
    rng = np.random.default_rng(7 * M + N + K)
    A = rng.standard_normal((M, K)) * np.exp(-np.arange(K) / 300.0)[None, :]
    B = rng.standard_normal((N, K)) * 10.0 ** rng.uniform(-3, 3, size=(N, 1))
    C = np.empty((M, N))
    with lib_context() as ctx:                   # float64 context: digits select the engine
        ctx.tc_gemm(A, B, C, digits=7)
    assert np.array_equal(C, fx_model(A, B, ns=7))
    ref = A @ B.T
    amax, bmax = np.abs(A).max(axis=1)[:, None], np.abs(B).max(axis=1)[None, :]
    assert np.all(np.abs(C - ref) <= K * 2.0 ** -52 * amax * bmax)
    assert np.abs(C - ref).max() / np.abs(ref).max() < 1e-14


@pytest.mark.parametrize("prec,tol", [("bf16x3", 3e-5), ("tf32x3", 1.5e-5), ("bf16x6", 1.5e-5)])
def test_float_split_gemm_accuracy(prec, tol):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((150, 700))
    B = rng.standard_normal((90, 700))
    C = np.empty((150, 90))
    with lib_context(precision=prec) as ctx:
        ctx.tc_gemm(A, B, C)
    assert rel_max(C, A @ B.T) < tol


@pytest.mark.parametrize("nb,no,na,seed", [(24, 5, 72, 0), (71, 13, 150, 2), (100, 20, 300, 1)])
def test_bf16x10_pass_within_1meV(nb, no, na, seed):
    m = sy.molecule(nb, no, na, seed)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, ETA)
    nov = no * (nb - no)
    with lib_context(precision="bf16x10", eta=ETA) as ctx:
        load_mol(ctx, 0, m)
        om = np.empty(nov)
        ctx.rpa(0, om)
        sx = np.empty((nb, nb))
        sc = np.empty((nb, nb))
        ctx.sigma(0, sx, sc)
        eps = np.empty(nb)
        ctx.qs_step(0, eps)
    assert np.max(np.abs(om - r["Omega"])) < 1e-8
    assert rel_max(sx, r["sigma_x"]) < 1e-12
    assert rel_max(sc, r["sigma_c"]) < 1e-6
    assert np.max(np.abs(eps - r["eps_new"])) < 1.0 * MEV


def test_bf16x10_bench_size_within_1meV():
    m = sy.molecule(200, 40, 600, 1)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], 40, ETA)
    with lib_context(precision="bf16x10", eta=ETA) as ctx:
        load_mol(ctx, 0, m)
        sc = np.empty((200, 200))
        ctx.sigma(0, None, sc)
        eps = np.empty(200)
        ctx.qs_step(0, eps)
    assert rel_max(sc, r["sigma_c"]) < 1e-6
    assert np.max(np.abs(eps - r["eps_new"])) < 1.0 * MEV


@pytest.mark.parametrize("nb,no,na,seed", [(71, 13, 150, 2), (200, 40, 600, 1)])
def test_bf16x10_tc_ab_within_1meV(nb, no, na, seed):
    """(a) and (b) on the fixed-point engine too (MOLGW_FLAG_TC_AB): B and M to ~1e-9,
    Omega to ~1e-7 Ha, QP energies still within 1 meV."""
    from paper_2210_17093_gb300 import FLAG_TC_AB
    m = sy.molecule(nb, no, na, seed)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, ETA)
    nov = no * (nb - no)
    with lib_context(precision="bf16x10", eta=ETA, flags=FLAG_TC_AB) as ctx:
        load_mol(ctx, 0, m)
        M = np.empty(nov * nov)
        ctx.rpa_matrix(0, M)
        B = np.empty(na * nb * nb)
        ctx.fetch(0, "B", B)
        om = np.empty(nov)
        ctx.rpa(0, om)
        eps = np.empty(nb)
        ctx.qs_step(0, eps)
    print(f"nb={nb}: B {rel_max(B.reshape(na, nb, nb), r['B']):.2e} M {rel_max(M.reshape(nov, nov), r['M']):.2e} "
          f"Omega {np.max(np.abs(om - r['Omega'])):.2e} QP {np.max(np.abs(eps - r['eps_new'])) / MEV:.4f} meV")
    assert rel_max(B.reshape(na, nb, nb), r["B"]) < 1e-8
    assert rel_max(M.reshape(nov, nov), r["M"]) < 5e-8
    assert np.max(np.abs(om - r["Omega"])) < 1e-5
    assert np.max(np.abs(eps - r["eps_new"])) < 1.0 * MEV


def test_eig_tc_eigh_matches_float64():
    """MOLGW_FLAG_EIG_TC: the trailing updates on 7 digits and each mat-vec of the panel
    kernel (float64, tensor cores from 7-digit tile images, integer multiply-adds from
    53-bit images); eigenvalues to float64 accuracy and orthonormal residual-small
    eigenvectors.  n = 1100 runs the first panel's mat-vec on the tensor cores (trailing
    order >= 1024) and the integer one down to trailing order 256."""
    from paper_2210_17093_gb300 import FLAG_EIG_TC
    n = 1100
    rng = np.random.default_rng(11)
    X = rng.standard_normal((n, n))
    A = (X + X.T) / 2 + np.diag(np.linspace(-5, 5, n))
    ref = np.linalg.eigvalsh(A)
    out = {}
    for flags, kind in ((0, None), (FLAG_EIG_TC, "fp64"), (FLAG_EIG_TC, "tc"), (FLAG_EIG_TC, "int")):
        w = np.empty(n)
        Z = np.empty((n, n))
        with lib_context(flags=flags) as ctx:
            if kind is not None:
                ctx.set_panel_matvec(kind)
            ctx.eigh(np.ascontiguousarray(A), w, Z)
        out[(flags, kind)] = (w, Z)
    nrm = np.abs(ref).max()
    for flags, (w, Z) in out.items():
        assert np.max(np.abs(w - ref)) < 1e-12 * nrm, flags
        Zc = Z.reshape(n, n)
        # the layout the header states: Z[i][k] = component i of eigenvector k (columns),
        # each column's largest-magnitude entry positive
        assert np.abs(A @ Zc - Zc * w[None, :]).max() < 1e-10 * nrm, flags
        assert np.abs(Zc.T @ Zc - np.eye(n)).max() < 1e-12 * n, flags
        big = np.abs(Zc).argmax(axis=0)
        assert np.all(Zc[big, np.arange(n)] > 0), flags


@pytest.mark.parametrize("matvec", ["tc", "int"])
@pytest.mark.parametrize("prec,tol_ha", [("fp64", 1e-8), ("bf16x10", 1.0 * MEV)])
def test_eig_tc_pass(prec, tol_ha, matvec):
    from paper_2210_17093_gb300 import FLAG_EIG_TC
    nb, no, na = 100, 20, 300
    m = sy.molecule(nb, no, na, 1)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, ETA)
    nov = no * (nb - no)
    with lib_context(precision=prec, eta=ETA, flags=FLAG_EIG_TC) as ctx:
        ctx.set_panel_matvec(matvec)
        load_mol(ctx, 0, m)
        om = np.empty(nov)
        ctx.rpa(0, om)
        eps = np.empty(nb)
        ctx.qs_step(0, eps)
    assert np.max(np.abs(om - r["Omega"])) < 1e-8
    assert np.max(np.abs(eps - r["eps_new"])) < tol_ha
