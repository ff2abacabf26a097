"""The GPU parity bars are tight enough to catch the plausible mistakes.

For every mistake planted in the oracle by ``test_oracle_mutations.py`` (a dropped
factor, a flipped sign, a wrong index range, a transposed product), a kernel making the
same mistake would move at least one output that the GPU parity tests compare with
the oracle -- Omega, Sigma_x, Sigma_c, J, the updated energies and occupied projector
over two iterations, the G0W0 energies and Z, per spin for an open shell -- by more
than 100 times that output's bar (float64 bars of ``tests/test_gpu_*.py``).  Run on the
small workload of the GPU tests (n_basis 24, n_occ 5, n_aux 72, seed 0).
"""
import numpy as np
import pytest

import synthetic as sy
import test_oracle_mutations as TM
from oracle import qsgw

ETA = sy.ETA
BAR_ABS = 1e-8      # Omega, energies, projectors, Z (Ha or dimensionless)
BAR_REL = 1e-6      # Sigma_x, Sigma_c, relative to their maximum
MARGIN = 100.0


def _mol():
    m = sy.molecule(24, 5, 72, 0)
    rng = np.random.default_rng(7)
    Cdn, _ = np.linalg.qr(m["C"] + 0.3 * rng.standard_normal((24, 24)))
    edn = np.sort(m["eps"] + 0.2 * rng.standard_normal(24))
    return m, Cdn, edn


def _proj(C, no):
    return C[:, :no] @ C[:, :no].T


def outputs():
    """Every compared output: name -> (array, 'abs' | 'rel')."""
    m, Cdn, edn = _mol()
    L, eps, C, no = m["L"], m["eps"], m["C"], 5
    out = {}
    its = qsgw.qsgw_iterations(L, eps, C, no, ETA, 2)
    out["gw.Omega"] = (its[0]["Omega"], "abs")
    out["gw.sigma_x"] = (its[0]["sigma_x"], "rel")
    out["gw.sigma_c"] = (its[0]["sigma_c"], "rel")
    out["gw.J"] = (its[0]["J"], "rel")
    for k in (0, 1):
        out[f"gw.eps{k}"] = (its[k]["eps_new"], "abs")
        out[f"gw.P{k}"] = (_proj(its[k]["C_new"], no), "abs")
    mp = qsgw.qsmp2_iterations(L, eps, C, no, ETA, 2)
    out["mp2.sigma_c"] = (mp[0]["sigma_c"], "rel")
    for k in (0, 1):
        out[f"mp2.eps{k}"] = (mp[k]["eps_new"], "abs")
    g = qsgw.g0w0_pass(L, eps, C, no, ETA)
    out["g0w0.eps_qp"] = (g["eps_qp"], "abs")
    out["g0w0.Z"] = (g["Z"], "abs")
    o = qsgw.qsgw_pass_open(L, (eps, edn), (C, Cdn), (5, 4), ETA)
    out["open.Omega"] = (o["Omega"], "abs")
    for k, sp in enumerate(o["spin"]):
        out[f"open.sigma_c{k}"] = (sp["sigma_c"], "rel")
        out[f"open.sigma_x{k}"] = (sp["sigma_x"], "rel")
        out[f"open.J{k}"] = (sp["J"], "rel")
        out[f"open.eps{k}"] = (sp["eps_new"], "abs")
    return out


@pytest.fixture(scope="module")
def reference():
    return outputs()


def _exceedance(ref, got):
    worst, where = 0.0, None
    for name, (a, kind) in ref.items():
        b = got[name][0]
        if a.shape != b.shape:
            return np.inf, name
        d = float(np.max(np.abs(b - a)))
        if kind == "rel":
            d /= max(float(np.max(np.abs(a))), 1e-300)
        r = d / (BAR_REL if kind == "rel" else BAR_ABS)
        if not np.isfinite(r) or r > worst:
            worst, where = (np.inf if not np.isfinite(r) else r), name
    return worst, where


def test_unmutated_oracle_is_reproducible(reference):
    worst, where = _exceedance(reference, outputs())
    assert worst == 0.0, (worst, where)


@pytest.mark.parametrize("mutant", sorted(TM.MUTANTS))
def test_mistake_exceeds_a_parity_bar(mutant, reference, monkeypatch):
    for attr, fn in TM.MUTANTS[mutant]().items():
        monkeypatch.setattr(qsgw, attr, fn)
    try:
        got = outputs()
    except FloatingPointError:
        return          # the pass refuses the input (the GPU latches MOLGW_E_NUMERIC)
    worst, where = _exceedance(reference, got)
    assert worst > MARGIN, (mutant, worst, where)
