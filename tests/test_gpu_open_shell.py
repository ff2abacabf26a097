"""Open-shell (sigma-resolved) qsGW on the float64 path against the oracle
(``oracle.qsgw.qsgw_pass_open``), molgw_b200_set_orbitals_open."""
import numpy as np
import pytest

import synthetic as sy
from helpers import lib_context, rel_max, to_dev
from oracle import qsgw

pytestmark = pytest.mark.gpu
ETA = sy.ETA


def open_molecule(nb, no_up, no_dn, na, seed):
    m = sy.molecule(nb, no_up, na, seed)
    rng = np.random.default_rng(1000 + seed)
    Cdn, _ = np.linalg.qr(m["C"] + 0.3 * rng.standard_normal((nb, nb)))
    edn = np.sort(m["eps"] + 0.2 * rng.standard_normal(nb))
    return m["L"], (m["eps"], edn), (m["C"], Cdn), (no_up, no_dn)


def load_open(ctx, mol, L, epss, Cs, nos, h_core=None):
    nb, na = Cs[0].shape[0], L.shape[0]
    ctx.set_ri(mol, nb, na, to_dev(L))
    ctx.set_orbitals_open(mol, nos[0], nos[1], to_dev(epss[0]), to_dev(epss[1]), to_dev(Cs[0]), to_dev(Cs[1]),
                          None if h_core is None else to_dev(h_core))


def proj(C, no):
    return C[:, :no] @ C[:, :no].T


@pytest.mark.parametrize("nb,nos,na,seed", [
    (24, (5, 4), 72, 40),     # one more spin-up electron
    (71, (13, 11), 150, 41),  # several tiles, ragged tails
    (30, (1, 0), 60, 42),     # one electron
    (33, (32, 30), 50, 43),   # nearly full channels
])
def test_open_shell_pass_against_oracle(nb, nos, na, seed):
    L, epss, Cs, nos = open_molecule(nb, nos[0], nos[1], na, seed)
    r = qsgw.qsgw_pass_open(L, epss, Cs, nos, ETA)
    n = sum(no * (nb - no) for no in nos)
    with lib_context() as ctx:
        load_open(ctx, 0, L, epss, Cs, nos)
        om = np.empty(n)
        ctx.rpa(0, om)
        sx = np.empty((2, nb, nb))
        sc = np.empty((2, nb, nb))
        ctx.sigma(0, sx, sc)
        J = np.empty((2, nb, nb))
        ctx.fetch(0, "J", J)
        eps = np.empty((2, nb))
        C = np.empty((2, nb, nb))
        ctx.qs_step(0, eps, C)
    assert np.max(np.abs(om - r["Omega"])) < 1e-8
    for k in (0, 1):
        sp = r["spin"][k]
        assert rel_max(sx[k], sp["sigma_x"]) < 1e-12 or np.max(np.abs(sp["sigma_x"])) == 0.0
        assert rel_max(J[k], sp["J"]) < 1e-12
        assert rel_max(sc[k], sp["sigma_c"]) < 1e-10
        assert np.max(np.abs(eps[k] - sp["eps_new"])) < 1e-8
        assert np.max(np.abs(proj(C[k], nos[k]) - proj(sp["C_new"], nos[k]))) < 1e-8


def test_equal_channels_match_the_closed_shell_gpu_path():
    nb, no, na = 40, 8, 96
    m = sy.molecule(nb, no, na, 44)
    with lib_context() as ctx:
        ctx.set_ri(0, nb, na, to_dev(m["L"]))
        ctx.set_orbitals(0, no, to_dev(m["eps"]), to_dev(m["C"]))
        e_closed = np.empty(nb)
        ctx.qs_step(0, e_closed)
        load_open(ctx, 0, m["L"], (m["eps"], m["eps"]), (m["C"], m["C"]), (no, no))
        e_open = np.empty((2, nb))
        ctx.qs_step(0, e_open)
    assert np.max(np.abs(e_open[0] - e_closed)) < 1e-9
    assert np.max(np.abs(e_open[1] - e_closed)) < 1e-9


def test_open_shell_second_step_from_the_gpu_state():
    nb, na = 40, 96
    L, epss, Cs, nos = open_molecule(nb, 8, 7, na, 45)
    with lib_context() as ctx:
        load_open(ctx, 0, L, epss, Cs, nos)
        ctx.qs_step(0)
        eps_in, C_in, h_in = np.empty((2, nb)), np.empty((2, nb, nb)), np.empty((2, nb, nb))
        ctx.fetch(0, "eps", eps_in)
        ctx.fetch(0, "C", C_in)
        ctx.fetch(0, "h_mo", h_in)
        eps = np.empty((2, nb))
        ctx.qs_step(0, eps)
    r = qsgw.qsgw_pass_open(L, (eps_in[0], eps_in[1]), (C_in[0], C_in[1]), nos, ETA, h_mos=(h_in[0], h_in[1]))
    for k in (0, 1):
        assert np.max(np.abs(eps[k] - r["spin"][k]["eps_new"])) < 1e-8


def test_open_and_closed_molecules_in_one_batch():
    nb, na = 36, 80
    L, epss, Cs, nos = open_molecule(nb, 7, 6, na, 46)
    mc = sy.batch_molecule(140)
    solo = []
    with lib_context() as ctx:
        load_open(ctx, 0, L, epss, Cs, nos)
        e = np.empty((2, nb))
        ctx.qs_step(0, e)
        solo.append(e)
    with lib_context() as ctx:
        ctx.set_ri(0, mc["n_basis"], mc["n_aux"], to_dev(mc["L"]))
        ctx.set_orbitals(0, mc["n_occ"], to_dev(mc["eps"]), to_dev(mc["C"]))
        e = np.empty(mc["n_basis"])
        ctx.qs_step(0, e)
        solo.append(e)
    with lib_context(max_mols=2, lanes=1) as ctx:
        load_open(ctx, 0, L, epss, Cs, nos)
        ctx.set_ri(1, mc["n_basis"], mc["n_aux"], to_dev(mc["L"]))
        ctx.set_orbitals(1, mc["n_occ"], to_dev(mc["eps"]), to_dev(mc["C"]))
        ctx.qs_step(-1)
        ctx.sync()
        e0 = np.empty((2, nb))
        ctx.fetch(0, "eps", e0)
        e1 = np.empty(mc["n_basis"])
        ctx.fetch(1, "eps", e1)
    assert np.array_equal(e0, solo[0])
    assert np.array_equal(e1, solo[1])


def test_open_shell_argument_and_state_errors():
    from paper_2210_17093_gb300 import MolgwError
    nb, na = 24, 72
    L, epss, Cs, nos = open_molecule(nb, 5, 4, na, 47)
    with lib_context(precision="bf16x3") as ctx:
        with pytest.raises(MolgwError):
            load_open(ctx, 0, L, epss, Cs, nos)
    with lib_context() as ctx:
        with pytest.raises(MolgwError):
            load_open(ctx, 0, L, epss, Cs, (0, 0))
        load_open(ctx, 0, L, epss, Cs, nos)
        with pytest.raises(MolgwError):
            ctx.g0w0(0, np.empty(nb))
        ctx.qs_step(0)
        with pytest.raises(MolgwError):
            ctx.fetch(0, "eps_qp", np.empty(nb))
        # set_orbitals makes the molecule closed again
        m = sy.molecule(nb, 5, na, 47)
        ctx.set_orbitals(0, 5, to_dev(m["eps"]), to_dev(m["C"]))
        e = np.empty(nb)
        ctx.qs_step(0, e)


def test_open_shell_graph_replay_and_autotune():
    """Three steps replayed from a captured graph equal three eager steps; autotuning a
    context that holds an open-shell molecule puts both spin channels back."""
    nb, na = 36, 80
    L, epss, Cs, nos = open_molecule(nb, 7, 6, na, 48)
    out = []
    for flags, tune in ((0, False), (4, False), (0, True)):
        with lib_context(flags=flags) as ctx:
            load_open(ctx, 0, L, epss, Cs, nos)
            if tune:
                ctx.autotune()
            for _ in range(3):
                ctx.qs_step(-1)
            ctx.sync()
            e = np.empty((2, nb))
            ctx.fetch(0, "eps", e)
            out.append(e)
    assert np.array_equal(out[0], out[1])
    assert np.max(np.abs(out[2] - out[0])) < 1e-8


@pytest.mark.parametrize("flags", [0, 16, 48])
@pytest.mark.parametrize("nb,nos,na,seed", [(24, (5, 4), 72, 40), (71, (13, 11), 150, 41)])
def test_open_shell_fixed_point_within_1mev(flags, nb, nos, na, seed):
    """BF16X10: (d)+(e) per spin on the fixed-point engine; with MOLGW_FLAG_TC_AB (16)
    also (a) per spin and (b); with MOLGW_FLAG_EIG_TC (32) the eigensolver's trailing
    updates on the 7-digit engine."""
    L, epss, Cs, nos = open_molecule(nb, nos[0], nos[1], na, seed)
    r = qsgw.qsgw_pass_open(L, epss, Cs, nos, ETA)
    with lib_context(precision="bf16x10", flags=flags) as ctx:
        load_open(ctx, 0, L, epss, Cs, nos)
        eps = np.empty((2, nb))
        ctx.qs_step(0, eps)
    for k in (0, 1):
        assert np.max(np.abs(eps[k] - r["spin"][k]["eps_new"])) < 3.675e-5
