"""Parity at the large workloads, where the kernels take their large-size paths.

* 400/80/1200 (25,600 transitions, seed 4): one pass from the input orbitals against
  the oracle's stored values (tests/golden/qsgw_nb400_no80_na1200_seed4.npz, written
  by tests/golden/make_golden.py C from oracle/ only).  n_aux = 1200 spans two
  1024-wide scale groups of the fixed-point residue GEMM (the multi-group path).
  Float64: Omega and the QP energies within 1e-8 Ha; BF16X10 with TC_AB: within
  1 meV; Sigma_x and Sigma_c within 1e-6 of their maximum for both.
* 600/120/1800 (57,600 transitions, M 26.5 GB, n^2 > 2^31), seed 7, BF16X10 with
  TC_AB and EIG_TC: Sigma_x and J element by element against the oracle (from the
  oracle's own B), the eight largest Omega against a Lanczos solve of the oracle's
  matrix-free Casida operator, sum Omega^2 = tr M, Omega_min >= min D, Sigma_c
  symmetric.
* The eigensolver at n = 46,400 (n^2 > 2^31 elements) on a dense matrix of known
  spectrum, A = H diag(lam) H with H = I - 2 u u^T: every eigenvalue, and residuals
  and orthogonality of a sample of eigenvectors computed on the host in O(n) each.
"""
import os

import numpy as np
import pytest

import synthetic as sy
from helpers import lib_context, rel_max, to_dev
from oracle import qsgw

pytestmark = pytest.mark.gpu
HA_MEV = 27211.386
MEV = 1.0 / HA_MEV
GOLDEN_C = os.path.join(os.path.dirname(__file__), "golden", "qsgw_nb400_no80_na1200_seed4.npz")
FLAG_TC_AB, FLAG_EIG_TC = 16, 32


@pytest.fixture(scope="module")
def config_c():
    if not os.path.exists(GOLDEN_C):
        pytest.fail("stored oracle values missing: run python tests/golden/make_golden.py C")
    g = dict(np.load(GOLDEN_C))
    nb, no, na, seed = (int(x) for x in g["workload"])
    return sy.molecule(nb, no, na, seed), g


def _pass(m, **kw):
    nb, no, na = m["n_basis"], m["n_occ"], m["n_aux"]
    n = no * (nb - no)
    with lib_context(**kw) as ctx:
        ctx.set_ri(0, nb, na, to_dev(m["L"]))
        ctx.set_orbitals(0, no, to_dev(m["eps"]), to_dev(m["C"]))
        eps = np.empty(nb)
        ctx.qs_step(0, eps)
        om, sx, sc = np.empty(n), np.empty((nb, nb)), np.empty((nb, nb))
        ctx.fetch(0, "Omega", om)
        ctx.fetch(0, "sigma_x", sx)
        ctx.fetch(0, "sigma_c", sc)
    return om, sx, sc, eps


@pytest.mark.parametrize("precision,flags,bar", [("fp64", 0, 1e-8), ("bf16x10", FLAG_TC_AB, MEV)])
def test_config_c_pass_against_stored_oracle(config_c, precision, flags, bar):
    m, g = config_c
    om, sx, sc, eps = _pass(m, precision=precision, flags=flags)
    iu = np.triu_indices(m["n_basis"])
    assert np.max(np.abs(om - g["Omega"])) <= bar
    assert np.max(np.abs(eps - g["eps_new"])) <= bar
    assert rel_max(sx[iu], g["sigma_x_upper"]) <= 1e-6
    assert rel_max(sc[iu], g["sigma_c_upper"]) <= 1e-6
    assert np.min(om) >= float(g["min_D"])
    assert np.sum(om * om) == pytest.approx(float(g["trace_M"]), rel=1e-9 if precision == "fp64" else 1e-6)


def test_config_e_pass_sampled_against_oracle():
    import scipy.sparse.linalg as sla
    nb, no, na, seed = 600, 120, 1800, 7
    m = sy.molecule(nb, no, na, seed)
    n = no * (nb - no)
    with lib_context(precision="bf16x10", flags=FLAG_TC_AB | FLAG_EIG_TC) as ctx:
        ctx.set_ri(0, nb, na, to_dev(m["L"]))
        ctx.set_orbitals(0, no, to_dev(m["eps"]), to_dev(m["C"]))
        eps = np.empty(nb)
        ctx.qs_step(0, eps)
        om, sx, sc, J = np.empty(n), np.empty((nb, nb)), np.empty((nb, nb)), np.empty((nb, nb))
        ctx.fetch(0, "Omega", om)
        ctx.fetch(0, "sigma_x", sx)
        ctx.fetch(0, "sigma_c", sc)
        ctx.fetch(0, "J", J)
    # the oracle's own B, Sigma_x, J and Casida operator for the same input orbitals
    B = qsgw.ri_mo_transform(m["L"], m["C"])
    assert rel_max(sx, qsgw.sigma_x(B, no)) <= 1e-6
    assert rel_max(J, qsgw.hartree(B, no)) <= 1e-6
    apply, D = qsgw.casida_M_apply(B, m["eps"], no)
    op = sla.LinearOperator((n, n), matvec=apply, matmat=apply, dtype=np.float64)
    top = np.sort(sla.eigsh(op, k=8, which="LA", tol=1e-13, return_eigenvectors=False))
    assert np.max(np.abs(np.sort(om)[-8:] - np.sqrt(top))) <= MEV
    tr_m = float(np.sum(D * D) + 4.0 * np.sum(D * np.sum(B[:, :no, no:].reshape(na, n) ** 2, axis=0)))
    assert np.sum(om * om) == pytest.approx(tr_m, rel=1e-6)
    assert np.all(np.diff(om) >= 0.0) and np.min(om) >= np.min(D) - 1e-4
    assert np.max(np.abs(sc - sc.T)) <= 1e-12 * np.max(np.abs(sc))
    assert np.all(np.isfinite(eps)) and np.all(np.diff(eps) >= 0.0)


def _known_spectrum(n, seed):
    """A = H diag(lam) H, H = I - 2 u u^T (|u| = 1): eigenvalues lam, eigenvectors H e_k."""
    rng = np.random.default_rng(seed)
    # spacing 2/n with jitter below a quarter of it: gaps >= 1/n keep the eigenvectors
    # well conditioned (a uniform random spectrum would put some pairs 1e-9 apart)
    lam = -1.0 + 2.0 * (np.arange(n) + 0.5 + rng.uniform(-0.25, 0.25, n)) / n
    u = rng.standard_normal(n)
    u /= np.linalg.norm(u)
    return lam, u


def _apply_known(lam, u, z):
    """A z for A = H diag(lam) H in O(n)."""
    hz = z - 2.0 * u * (u @ z)
    y = lam * hz
    return y - 2.0 * u * (u @ y)


@pytest.mark.parametrize("flags", [0, FLAG_EIG_TC])
def test_eigensolver_beyond_2_31_elements(flags):
    torch = pytest.importorskip("torch")
    n = 46400                                   # n^2 = 2.15e9 > 2^31
    lam, u = _known_spectrum(n, 11)
    ud = torch.from_numpy(u).cuda()
    ld = torch.from_numpy(lam).cuda()
    lu = ld * ud
    c = float((ud * lu).sum())
    A = -2.0 * torch.outer(ud, lu)
    A -= 2.0 * torch.outer(lu, ud)
    A += 4.0 * c * torch.outer(ud, ud)
    A.diagonal().add_(ld)
    del lu
    want_vectors = bool(flags & FLAG_EIG_TC)   # the float64 back-transformation would take minutes
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    Z = torch.empty((n, n), dtype=torch.float64, device="cuda") if want_vectors else None
    with lib_context(flags=flags) as ctx:
        ctx.eigh(A, w, Z)
        ctx.sync()
    del A
    wh = w.cpu().numpy()
    assert np.max(np.abs(wh - lam)) <= 1e-12 * np.sqrt(n)
    assert abs(np.sum(wh) - np.sum(lam)) <= 1e-9
    if want_vectors:
        ks = np.unique(np.concatenate([np.arange(4), n - 1 - np.arange(4),
                                       np.random.default_rng(3).integers(0, n, 56)]))
        zs = Z[:, torch.from_numpy(ks).cuda()].cpu().numpy()       # columns = eigenvectors
        del Z
        for j, k in enumerate(ks):
            z = zs[:, j]
            assert np.linalg.norm(_apply_known(lam, u, z) - wh[k] * z) <= 1e-10
            e = -2.0 * u[k] * u
            e[k] += 1.0                           # H e_k, the exact eigenvector up to sign
            assert min(np.max(np.abs(z - e)), np.max(np.abs(z + e))) <= 1e-8
            assert np.abs(z).argmax() == np.abs(e).argmax() and z[np.abs(z).argmax()] > 0
        G = zs.T @ zs
        assert np.max(np.abs(G - np.eye(len(ks)))) <= 1e-10
