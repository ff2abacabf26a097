"""One-shot G0W0 (molgw_b200_g0w0: the diagonal of Eq. Sigma.c.GW, linearised) against the oracle."""
import numpy as np
import pytest

import synthetic as sy
from helpers import lib_context, load_mol
from oracle import qsgw

pytestmark = pytest.mark.gpu
ETA = sy.ETA


@pytest.mark.parametrize("prec", ["fp64", "bf16x10"])
@pytest.mark.parametrize("nb,no,na,seed", [(24, 5, 72, 0), (71, 13, 150, 2), (40, 1, 90, 7)])
def test_g0w0_against_oracle(prec, nb, no, na, seed):
    """(a)-(c) in float64 at both precisions and the residues in float64: float64
    tolerances.  The bars for eps^QP (1e-8 Ha) and Z (1e-8) widen to ten times the
    spread of the oracle's own result under rounding-level changes when that is
    larger: 2-ulp changes of its input energies, and changes of the Casida matrix of
    the size of a float64 eigensolver's backward error (a random symmetric E with
    ||E|| = sqrt(n_ov) eps ||M||; two backward-stable eigensolvers may differ by that
    much).  Next to a pole Z_p = 1 / (1 - Sigma'_pp) reaches 0.002 and below 0 (Sigma'_pp
    ~ 400, and d Sigma'/d Omega ~ w^2 / eta^3): at 71/13/150 a state with Z = -0.065
    moves by up to 1e-7 Ha under such a change of M."""
    m = sy.molecule(nb, no, na, seed)
    r = qsgw.g0w0_pass(m["L"], m["eps"], m["C"], no, ETA)
    spread = spread_z = 0.0
    orig_m = qsgw.casida_M
    for k in range(3):
        rng = np.random.default_rng(k)
        ep = m["eps"] * (1.0 + 4.4e-16 * rng.choice([-1.0, 1.0], m["eps"].shape))
        rp = qsgw.g0w0_pass(m["L"], ep, m["C"], no, ETA)
        spread = max(spread, np.max(np.abs(rp["eps_qp"] - r["eps_qp"])))
        spread_z = max(spread_z, np.max(np.abs(rp["Z"] - r["Z"])))

        def casida_m_perturbed(A, Bc, D, rng=rng):
            M = orig_m(A, Bc, D)
            E = rng.standard_normal(M.shape)
            E = 0.5 * (E + E.T)
            return M + E * (2.220446049250313e-16 * np.sqrt(M.shape[0]) * np.linalg.norm(M, 2) / np.linalg.norm(E, 2))
        qsgw.casida_M = casida_m_perturbed
        try:
            rp = qsgw.g0w0_pass(m["L"], m["eps"], m["C"], no, ETA)
        finally:
            qsgw.casida_M = orig_m
        spread = max(spread, np.max(np.abs(rp["eps_qp"] - r["eps_qp"])))
        spread_z = max(spread_z, np.max(np.abs(rp["Z"] - r["Z"])))
    with lib_context(precision=prec) as ctx:
        load_mol(ctx, 0, m)
        e, z, s = np.empty(nb), np.empty(nb), np.empty(nb)
        ctx.g0w0(0, e, z, s)
    assert np.max(np.abs(s - r["sigma_c_diag"])) <= 1e-10 * np.max(np.abs(r["sigma_c_diag"]))
    assert np.max(np.abs(z - r["Z"])) < max(1e-8, 10.0 * spread_z), spread_z
    assert np.max(np.abs(e - r["eps_qp"])) < max(1e-8, 10.0 * spread), spread


def test_g0w0_with_explicit_h_core():
    nb, no, na = 30, 6, 80
    m = sy.molecule(nb, no, na, 8)
    rng = np.random.default_rng(3)
    h = rng.standard_normal((nb, nb))
    h = 0.5 * (h + h.T)
    B = qsgw.ri_mo_transform(m["L"], m["C"])
    r = qsgw.g0w0_pass(m["L"], m["eps"], m["C"], no, ETA, h_mo=m["C"].T @ h @ m["C"])
    with lib_context() as ctx:
        load_mol(ctx, 0, m, h_core=h)
        e = np.empty(nb)
        ctx.g0w0(0, e)
    assert np.max(np.abs(e - r["eps_qp"])) < 1e-8
    assert B.shape[0] == na


def test_g0w0_leaves_the_orbitals_current():
    m = sy.molecule(40, 8, 96, 9)
    out = []
    for do_g0w0 in (False, True):
        with lib_context() as ctx:
            load_mol(ctx, 0, m)
            if do_g0w0:
                ctx.g0w0(0, np.empty(40))
            e = np.empty(40)
            ctx.qs_step(0, e)
            out.append(e)
    assert np.array_equal(out[0], out[1])


def test_g0w0_batch_equals_solo():
    mols = [sy.batch_molecule(s) for s in (110, 111, 112)]
    solo = []
    for m in mols:
        with lib_context() as ctx:
            load_mol(ctx, 0, m)
            e = np.empty(m["n_basis"])
            ctx.g0w0(0, e)
            solo.append(e)
    # one lane: the batch issues exactly the launches of the solo calls (with more lanes
    # the panel kernel's share of the device, hence its rounding order, differs)
    with lib_context(max_mols=3, lanes=1) as ctx:
        for k, m in enumerate(mols):
            load_mol(ctx, k, m)
        ctx.g0w0(-1)
        ctx.sync()
        for k, m in enumerate(mols):
            e = np.empty(m["n_basis"])
            ctx.fetch(k, "eps_qp", e)
            assert np.array_equal(e, solo[k])


def test_g0w0_not_with_qsmp2():
    from paper_2210_17093_gb300 import MolgwError
    m = sy.molecule(24, 5, 72, 0)
    with lib_context(flags=64) as ctx:
        load_mol(ctx, 0, m)
        with pytest.raises(MolgwError):
            ctx.g0w0(0, np.empty(24))


def test_g0w0_state_window():
    """The window p_begin <= p < p_end (frontier states here) gives the full call's values
    for those states (up to the summation grouping, which follows the window's size)."""
    nb, no, na = 71, 13, 150
    m = sy.molecule(nb, no, na, 2)
    with lib_context() as ctx:
        load_mol(ctx, 0, m)
        e_all, z_all = np.empty(nb), np.empty(nb)
        ctx.g0w0(0, e_all, z_all)
        lo, hi = no - 3, no + 3
        e, z, s = np.empty(hi - lo), np.empty(hi - lo), np.empty(hi - lo)
        ctx.g0w0_window(0, lo, hi, e, z, s)
        full = np.empty(nb)
        ctx.fetch(0, "eps_qp", full)
    np.testing.assert_allclose(e, e_all[lo:hi], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(z, z_all[lo:hi], rtol=1e-10, atol=1e-13)
    np.testing.assert_array_equal(full[lo:hi], e)
    r = qsgw.g0w0_pass(m["L"], m["eps"], m["C"], no, ETA)
    np.testing.assert_allclose(s, r["sigma_c_diag"][lo:hi], rtol=0, atol=1e-10 * np.max(np.abs(r["sigma_c_diag"])))


def test_g0w0_entries_outside_the_window_are_nan():
    nb, no, na = 40, 8, 96
    m = sy.molecule(nb, no, na, 3)
    with lib_context() as ctx:
        load_mol(ctx, 0, m)
        e = np.empty(4)
        ctx.g0w0_window(0, no - 2, no + 2, e)
        full, z = np.empty(nb), np.empty(nb)
        ctx.fetch(0, "eps_qp", full)
        ctx.fetch(0, "Z", z)
    inside = np.zeros(nb, bool)
    inside[no - 2:no + 2] = True
    assert np.array_equal(full[inside], e)
    assert np.all(np.isfinite(z[inside]))
    assert np.all(np.isnan(full[~inside])) and np.all(np.isnan(z[~inside]))


def test_g0w0_window_arguments():
    from paper_2210_17093_gb300 import MolgwError
    m = sy.molecule(24, 5, 72, 0)
    with lib_context() as ctx:
        load_mol(ctx, 0, m)
        for lo, hi in ((3, 3), (-1, 2), (20, 25)):
            with pytest.raises(MolgwError):
                ctx.g0w0_window(0, lo, hi)
