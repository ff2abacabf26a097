"""Host logic of batches: the lane plan (molgw_b200_plan_batch), no GPU needed.

The library's planner is the one ``mol = -1`` uses.  It is checked against a plain
restatement of its cost model and of longest-processing-time-first scheduling,
against brute force on tiny batches (the LPT makespan bound 4/3 - 1/(3m) of the
optimum), and for its argument checks.
"""
import itertools

import numpy as np
import pytest

MAX_LANES, DEFAULT_LANES = 16, 8


@pytest.fixture(scope="module")
def plan():
    from paper_2210_17093_gb300 import build, native
    build.build()
    native.load()
    return native.plan_batch


def cost(nb, na, nu, nd=-1, mp2=False):
    nov = nu * (nb - nu) + (nd * (nb - nd) if nd >= 0 else 0)
    if mp2:
        return 4.0 * nb * nb * nov * na + 2.0 * nb ** 3 * nov
    return float(nov) ** 3 + (2.0 if nd >= 0 else 1.0) * 2.0 * nb * nb * nov * na


def lpt(costs, lanes):
    m = max(1, min(lanes, len(costs)))
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0.0] * m
    lane_of, slot = [0] * len(costs), [0] * len(costs)
    count = [0] * m
    for k in order:
        j = min(range(m), key=lambda x: (load[x], x))
        lane_of[k], slot[k] = j, count[j]
        count[j] += 1
        load[j] += costs[k]
    return lane_of, slot


def batch(seed, n):
    rng = np.random.default_rng(seed)
    nb = rng.integers(40, 161, size=n)
    return nb, 3 * nb, np.maximum(1, np.rint(nb / 5).astype(int))


@pytest.mark.parametrize("seed,n,lanes", [(0, 64, 0), (1, 64, 12), (2, 5, 8), (3, 40, 16), (4, 33, 40), (5, 1, 3)])
def test_matches_lpt_restatement(plan, seed, n, lanes):
    nb, na, no = batch(seed, n)
    lane_of, slot = plan(nb, na, no, lanes=lanes)
    want = min(lanes if lanes > 0 else DEFAULT_LANES, MAX_LANES)
    c = [cost(int(b), int(a), int(o)) for b, a, o in zip(nb, na, no)]
    wl, ws = lpt(c, want)
    assert lane_of.tolist() == wl
    assert slot.tolist() == ws


def test_plan_is_a_partition_in_decreasing_cost(plan):
    nb, na, no = batch(7, 50)
    lane_of, slot = plan(nb, na, no, lanes=6)
    c = np.array([cost(int(b), int(a), int(o)) for b, a, o in zip(nb, na, no)])
    assert set(lane_of.tolist()) == set(range(6))
    for j in range(6):
        mine = np.flatnonzero(lane_of == j)
        order = mine[np.argsort(slot[mine])]
        assert sorted(slot[mine].tolist()) == list(range(mine.size))
        assert np.all(np.diff(c[order]) <= 0)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("lanes", [2, 3])
def test_lpt_makespan_bound_against_brute_force(plan, seed, lanes):
    rng = np.random.default_rng(100 + seed)
    n = 7
    nb = rng.integers(6, 40, size=n)
    na = rng.integers(1, 3 * nb + 1)
    no = rng.integers(1, nb)
    c = [cost(int(b), int(a), int(o)) for b, a, o in zip(nb, na, no)]
    lane_of, _ = plan(nb, na, no, lanes=lanes)
    span = max(sum(c[k] for k in range(n) if lane_of[k] == j) for j in range(lanes))
    best = min(max(sum(c[k] for k in range(n) if a[k] == j) for j in range(lanes))
               for a in itertools.product(range(lanes), repeat=n))
    assert span <= (4.0 / 3.0 - 1.0 / (3 * lanes)) * best * (1 + 1e-12)


def test_open_shell_and_qsmp2_cost_models(plan):
    # the same transition count: the open shell has two residue channels and goes first
    nb, na = 50, 150
    lane_of, slot = plan([nb, nb], [na, na], [10, 10], n_occ_dn=[-1, 0], lanes=1)
    assert slot.tolist() == [1, 0]
    # qsMP2: the nb^2 n_ov na terms dominate, not n_ov^3
    nbs, nas, nos = [100, 60], [60, 1800], [50, 20]
    assert cost(100, 60, 50) > cost(60, 1800, 20) and cost(100, 60, 50, mp2=True) < cost(60, 1800, 20, mp2=True)
    _, s_gw = plan(nbs, nas, nos, lanes=1)
    _, s_mp2 = plan(nbs, nas, nos, flags=64, lanes=1)
    assert s_gw.tolist() == [0, 1] and s_mp2.tolist() == [1, 0]


@pytest.mark.parametrize("args", [
    dict(n_basis=[1], n_aux=[3], n_occ=[1]),             # n_basis < 2
    dict(n_basis=[10], n_aux=[0], n_occ=[2]),            # n_aux < 1
    dict(n_basis=[10], n_aux=[30], n_occ=[10]),          # no empty orbital
    dict(n_basis=[10], n_aux=[30], n_occ=[0]),           # closed shell without electrons
    dict(n_basis=[10], n_aux=[30], n_occ=[0], n_occ_dn=[0]),   # open shell without electrons
    dict(n_basis=[10], n_aux=[30], n_occ=[3], n_occ_dn=[10]),
    dict(n_basis=[10], n_aux=[30], n_occ=[3], n_occ_dn=[2], flags=64),   # qsMP2 is closed shell
    dict(n_basis=[10], n_aux=[30], n_occ=[3], lanes=-1),
])
def test_argument_errors(plan, args):
    from paper_2210_17093_gb300 import MolgwError
    with pytest.raises(MolgwError):
        plan(**args)
