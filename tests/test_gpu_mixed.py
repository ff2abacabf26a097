"""Split-precision tensor-core path (stages (d), (e); optionally (a), (b)) against the oracle.

The tolerances are the accuracy this path achieves, not the float64 targets:
the tensor cores accumulate in float32 and lose about one float32 ulp per MMA
step, which leaves ~1e-5 relative error in Sigma_c (the unit-level check of
the engine sees ~1e-6 per 64-wide K block).  With Sigma_c entries of 20-100 Ha
on these strongly coupled synthetic inputs that is 3-50 meV in the
quasiparticle energies.  Omega_s stays at float64 accuracy unless (a) and (b)
also run on the tensor cores (MOLGW_FLAG_TC_AB).
"""
import numpy as np
import pytest

import synthetic as sy
from helpers import lib_context, load_mol, rel_max
from oracle import qsgw

pytestmark = pytest.mark.gpu
ETA = sy.ETA


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "bf16x6"])
@pytest.mark.parametrize("nb,no,na,seed", [(24, 5, 72, 0), (71, 13, 150, 2)])
def test_mixed_sigma_and_qp(prec, nb, no, na, seed):
    m = sy.molecule(nb, no, na, seed)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, ETA)
    nov = no * (nb - no)
    with lib_context(precision=prec) as ctx:
        load_mol(ctx, 0, m)
        om = np.empty(nov)
        ctx.rpa(0, om)
        sx = np.empty((nb, nb))
        sc = np.empty((nb, nb))
        ctx.sigma(0, sx, sc)
        eps = np.empty(nb)
        ctx.qs_step(0, eps)
    assert np.max(np.abs(om - r["Omega"])) < 1e-8          # (a)-(c) in float64
    assert rel_max(sx, r["sigma_x"]) < 1e-12
    assert rel_max(sc, r["sigma_c"]) < 3e-5
    assert np.max(np.abs(eps - r["eps_new"])) < 2e-3        # Ha (~54 meV)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "bf16x6"])
def test_mixed_tc_ab(prec):
    """(a) and (b) on the tensor cores as well: B and M to ~1e-5 relative."""
    nb, no, na = 71, 13, 150
    m = sy.molecule(nb, no, na, 2)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, ETA)
    nov = no * (nb - no)
    with lib_context(precision=prec, flags=16) as ctx:
        load_mol(ctx, 0, m)
        M = np.empty(nov * nov)
        ctx.rpa_matrix(0, M)
        B = np.empty(na * nb * nb)
        ctx.fetch(0, "B", B)
        om = np.empty(nov)
        ctx.rpa(0, om)
    assert rel_max(B.reshape(na, nb, nb), r["B"]) < 2e-5
    assert rel_max(M.reshape(nov, nov), r["M"]) < 2e-5
    assert np.max(np.abs(om - r["Omega"])) < 1e-3


def test_mixed_bench_size():
    """nb=200: the self-energy on the tensor cores, eigensolvers in float64."""
    m = sy.molecule(200, 40, 600, 1)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], 40, ETA)
    with lib_context(precision="bf16x3") as ctx:
        load_mol(ctx, 0, m)
        sc = np.empty((200, 200))
        ctx.sigma(0, None, sc)
        eps = np.empty(200)
        ctx.qs_step(0, eps)
    assert rel_max(sc, r["sigma_c"]) < 3e-5
    assert np.max(np.abs(eps - r["eps_new"])) < 3e-3
