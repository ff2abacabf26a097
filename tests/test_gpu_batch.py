"""Batches (mol = -1) on concurrent lanes, and qs_step replayed from a captured
CUDA graph (MOLGW_FLAG_GRAPH), against the same calls issued one by one.

Molecules of the ragged batch: n_basis ~ U{40..160}, n_occ = round(n_basis/5),
n_aux = 3 n_basis (the batched workload of the qsGW pass, Sec. II.C)."""
import numpy as np
import pytest

import synthetic as sy
from helpers import lib_context, load_mol, rel_max

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9      # Ha; the lanes change only the summation order of the panel kernel


def fetch(ctx, k, m, item):
    nb, no = m["n_basis"], m["n_occ"]
    n = {"eps": nb, "C": nb * nb, "sigma_c": nb * nb, "Omega": no * (nb - no)}[item]
    out = np.empty(n)
    ctx.fetch(k, item, out)
    return out


def projector(C, no):
    C = C.reshape(int(round(np.sqrt(C.size))), -1)
    return C[:, :no] @ C[:, :no].T


def run_solo(m, precision="fp64", steps=1):
    with lib_context(stream=None, precision=precision, eta=sy.ETA) as ctx:
        load_mol(ctx, 0, m, device=False)
        for _ in range(steps):
            ctx.qs_step(0)
        return {it: fetch(ctx, 0, m, it) for it in ("eps", "C", "sigma_c", "Omega")}


def run_batch(mols, precision="fp64", lanes=0, steps=1, flags=0):
    with lib_context(stream=None, precision=precision, eta=sy.ETA, max_mols=len(mols), lanes=lanes,
                     flags=flags) as ctx:
        for k, m in enumerate(mols):
            load_mol(ctx, k, m, device=False)
        hist = []
        for _ in range(steps):
            ctx.qs_step(-1)
            hist.append([{it: fetch(ctx, k, m, it) for it in ("eps", "C", "sigma_c", "Omega")}
                         for k, m in enumerate(mols)])
        return hist, ctx.launch_count(), ctx.graph_replays()


def test_lanes_match_solo():
    mols = [sy.batch_molecule(s) for s in (100, 101, 104, 107, 108, 122)]
    hist, _, _ = run_batch(mols)
    for k, m in enumerate(mols):
        solo = run_solo(m)
        got = hist[0][k]
        no = m["n_occ"]
        assert np.max(np.abs(got["Omega"] - solo["Omega"])) < FP64_TOL, k
        assert np.max(np.abs(got["eps"] - solo["eps"])) < FP64_TOL, k
        assert rel_max(got["sigma_c"], solo["sigma_c"]) < 1e-8, k
        assert np.max(np.abs(projector(got["C"], no) - projector(solo["C"], no))) < 1e-8, k


def test_lanes_repeat_bitwise():
    mols = [sy.batch_molecule(s) for s in (102, 103, 105, 112)]
    a, _, _ = run_batch(mols, lanes=3)
    b, _, _ = run_batch(mols, lanes=3)
    for k in range(len(mols)):
        for it in ("eps", "C", "sigma_c", "Omega"):
            assert np.array_equal(a[0][k][it], b[0][k][it]), (k, it)


def test_more_lanes_than_molecules_and_empty_batch():
    from paper_2210_17093_gb300 import MolgwError
    m = sy.batch_molecule(108)
    hist, _, _ = run_batch([m], lanes=8)
    solo = run_solo(m)
    assert np.array_equal(hist[0][0]["eps"], solo["eps"])    # one molecule: one lane, as solo
    with lib_context(stream=None, max_mols=2) as ctx:
        with pytest.raises(MolgwError) as e:
            ctx.qs_step(-1)
        assert e.value.code == -2


@pytest.mark.parametrize("lanes", [1, 0])
def test_graph_replay_equals_eager(lanes):
    from paper_2210_17093_gb300 import FLAG_GRAPH
    mols = [sy.batch_molecule(s) for s in (101, 105, 107, 112, 123)]
    eager, n_eager, r_eager = run_batch(mols, lanes=lanes, steps=3)
    graph, n_graph, replays = run_batch(mols, lanes=lanes, steps=3, flags=FLAG_GRAPH)
    assert r_eager == 0
    # the first step derives h from the Hartree-Fock input (not the steady state);
    # the second is captured and launched, the third replays the graph
    assert replays == 2
    assert n_graph == n_eager
    for s in range(3):
        for k in range(len(mols)):
            for it in ("eps", "C", "sigma_c", "Omega"):
                assert np.array_equal(graph[s][k][it], eager[s][k][it]), (s, k, it)


def test_graph_replay_sees_new_inputs():
    """set_orbitals with h_core keeps the buffers (same sizes) and the steady state:
    the replayed graph must read the new orbitals."""
    from paper_2210_17093_gb300 import FLAG_GRAPH
    m1 = sy.molecule(48, 10, 96, 21)
    m2 = sy.molecule(48, 10, 96, 22)
    h = np.diag(m2["eps"])          # any symmetric h_core in the AO basis
    outs = []
    for flags in (0, FLAG_GRAPH):
        with lib_context(stream=None, eta=sy.ETA, flags=flags) as ctx:
            load_mol(ctx, 0, m1, device=False)
            ctx.qs_step(0)
            ctx.qs_step(0)                          # captured when graphs are on
            ctx.set_ri(0, 48, 96, np.ascontiguousarray(m2["L"]))
            ctx.set_orbitals(0, 10, np.ascontiguousarray(m2["eps"]), np.ascontiguousarray(m2["C"]),
                             np.ascontiguousarray(h))
            e = np.empty(48)
            ctx.qs_step(0, e)
            outs.append((e, ctx.graph_replays()))
    assert outs[1][1] >= 1
    assert np.array_equal(outs[0][0], outs[1][0])


def test_mixed_lanes_match_solo():
    mols = [sy.batch_molecule(s) for s in (100, 104, 108, 117)]
    hist, _, _ = run_batch(mols, precision="bf16x3")
    for k, m in enumerate(mols):
        solo = run_solo(m, precision="bf16x3")
        assert np.max(np.abs(hist[0][k]["eps"] - solo["eps"])) < 1e-7, k
        assert rel_max(hist[0][k]["sigma_c"], solo["sigma_c"]) < 1e-6, k


def test_autotune_restores_state_and_keeps_a_lane_count():
    """molgw_b200_autotune times trial steps and puts the orbitals back: the next step
    equals a step of a context fixed to the chosen lane count, bit for bit."""
    mols = [sy.batch_molecule(s) for s in (100, 101, 102, 104, 107, 110)]
    with lib_context(stream=None, eta=sy.ETA, max_mols=len(mols)) as ctx:
        for k, m in enumerate(mols):
            load_mol(ctx, k, m, device=False)
        lanes = ctx.autotune()
        assert ctx.lanes() == lanes and lanes in (4, 6)
        ctx.qs_step(-1)
        tuned = [fetch(ctx, k, m, "eps") for k, m in enumerate(mols)]
    hist, _, _ = run_batch(mols, lanes=lanes)
    for k in range(len(mols)):
        assert np.array_equal(tuned[k], hist[0][k]["eps"]), k


def test_bf16x10_tc_ab_lanes_match_solo():
    """The fixed-point path with (a) and (b) on the tensor cores too, as a batch on
    concurrent lanes (each lane carves its own operand arena) against solo runs."""
    from paper_2210_17093_gb300 import FLAG_TC_AB
    mols = [sy.batch_molecule(s) for s in (100, 105, 108, 122)]

    def solo(m):
        with lib_context(stream=None, precision="bf16x10", eta=sy.ETA, flags=FLAG_TC_AB) as ctx:
            load_mol(ctx, 0, m, device=False)
            ctx.qs_step(0)
            return fetch(ctx, 0, m, "eps")

    hist, _, _ = run_batch(mols, precision="bf16x10", flags=FLAG_TC_AB)
    for k, m in enumerate(mols):
        assert np.max(np.abs(hist[0][k]["eps"] - solo(m))) < 1e-7, k


def test_bf16x10_eig_tc_batch_graph_matches_solo():
    """The batch configuration of the bench: fixed point for (a), (b), (d), (e), the
    eigensolvers' trailing updates on the 7-digit engine, autotuned lanes, graph replay,
    against solo runs of each molecule (three steps)."""
    from paper_2210_17093_gb300 import FLAG_EIG_TC, FLAG_GRAPH, FLAG_TC_AB
    mols = [sy.batch_molecule(s) for s in (100, 105, 108, 122, 131)]
    flags = FLAG_TC_AB | FLAG_EIG_TC

    def solo(m):
        with lib_context(stream=None, precision="bf16x10", eta=sy.ETA, flags=flags) as ctx:
            load_mol(ctx, 0, m, device=False)
            ctx.qs_step(0)
            return fetch(ctx, 0, m, "eps")

    hist, _, replays = run_batch(mols, precision="bf16x10", flags=flags | FLAG_GRAPH, steps=3)
    assert replays >= 1
    for k, m in enumerate(mols):
        assert np.max(np.abs(hist[0][k]["eps"] - solo(m))) < 1e-7, k
