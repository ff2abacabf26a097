"""Checkpoint and resume: the state a qs_step leaves is (eps, C, h_MO).

Saving it with fetch and handing it to a fresh context through set_orbitals (h_core
= C h_MO C^T in the AO basis, since C is orthogonal) continues the trajectory: the
next iteration equals the one the uninterrupted context takes, up to the rounding of
the round trip of h through the AO basis.
"""
import numpy as np
import pytest

import synthetic as sy
from helpers import lib_context, load_mol, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,flags", [("fp64", 0), ("bf16x10", 16), ("fp64", 64)])
def test_resume_continues_the_trajectory(prec, flags):
    nb, no, na = 40, 8, 96
    m = sy.molecule(nb, no, na, 6)
    with lib_context(precision=prec, flags=flags) as ctx:
        load_mol(ctx, 0, m)
        ctx.qs_step(0)
        ctx.qs_step(0)
        eps, C, h = np.empty(nb), np.empty((nb, nb)), np.empty((nb, nb))
        ctx.fetch(0, "eps", eps)
        ctx.fetch(0, "C", C)
        ctx.fetch(0, "h_mo", h)
        e_cont, C_cont = np.empty(nb), np.empty((nb, nb))
        ctx.qs_step(0, e_cont, C_cont)
    h_ao = C @ h @ C.T
    with lib_context(precision=prec, flags=flags) as ctx2:
        ctx2.set_ri(0, nb, na, to_dev(m["L"]))
        ctx2.set_orbitals(0, no, to_dev(eps), to_dev(C), to_dev(h_ao))
        e_res, C_res = np.empty(nb), np.empty((nb, nb))
        ctx2.qs_step(0, e_res, C_res)
    scale = max(1.0, float(np.max(np.abs(e_cont))))
    assert np.max(np.abs(e_res - e_cont)) < 1e-9 * scale
    P = lambda X: X[:, :no] @ X[:, :no].T
    assert np.max(np.abs(P(C_res) - P(C_cont))) < 1e-8
