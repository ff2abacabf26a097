"""Failure detection without a GPU fault.

Device-detected error codes latched by the test hook molgw_b200_inject_fault travel
through the API the way a bounded wait that ran out would (returned by the next
synchronising call, then cleared), and the context stays usable.  With the bounds
lowered by molgw_b200_set_wait_limits the real device paths run out: the grid
barrier of the persistent panel kernel gives up after a few polls (every CTA
leaves the launch on the abort flag) and the bisection stops at its round cap; the
code reaches the caller and the next pass with the default bounds is bit-identical
to a clean one."""
import numpy as np
import pytest

import synthetic as sy
from helpers import lib_context, load_mol

pytestmark = pytest.mark.gpu
E_ARG, E_NOCONV, E_TIMEOUT, E_NUMERIC = -1, -5, -6, -7


@pytest.mark.parametrize("code", [E_TIMEOUT, E_NOCONV, E_NUMERIC])
def test_latched_code_reaches_the_caller_and_clears(code):
    from paper_2210_17093_gb300 import MolgwError
    m = sy.molecule(24, 5, 72, 0)
    with lib_context() as ref:
        load_mol(ref, 0, m)
        e_ref = np.empty(24)
        ref.qs_step(0)
        ref.qs_step(0, e_ref)
    with lib_context() as ctx:
        load_mol(ctx, 0, m)
        ctx.inject_fault(code)
        with pytest.raises(MolgwError) as ei:
            ctx.qs_step(0, np.empty(24))        # host output: synchronises, reads the word
        assert ei.value.code == code
        ctx.sync()                              # cleared
        e = np.empty(24)
        ctx.qs_step(0, e)                       # the context keeps working
    assert np.array_equal(e, e_ref)


def test_batch_call_reports_at_the_next_sync():
    from paper_2210_17093_gb300 import MolgwError
    mols = [sy.batch_molecule(s) for s in (130, 131)]
    with lib_context(max_mols=2) as ctx:
        for k, m in enumerate(mols):
            load_mol(ctx, k, m)
        ctx.inject_fault(E_TIMEOUT)
        ctx.qs_step(-1)                         # device outputs only: no synchronisation
        with pytest.raises(MolgwError) as ei:
            ctx.sync()
        assert ei.value.code == E_TIMEOUT
        ctx.sync()


def test_only_device_codes_can_be_injected():
    from paper_2210_17093_gb300 import MolgwError
    with lib_context() as ctx:
        for code in (E_ARG, 0, -3, 5):
            with pytest.raises(MolgwError) as ei:
                ctx.inject_fault(code)
            assert ei.value.code == E_ARG


@pytest.mark.parametrize("limits,code", [((0, -1), E_TIMEOUT), ((-1, 0), E_NOCONV)])
def test_device_bound_runs_out_and_the_context_recovers(limits, code):
    from paper_2210_17093_gb300 import MolgwError
    m = sy.molecule(24, 5, 72, 0)
    with lib_context() as ref:
        load_mol(ref, 0, m)
        e_ref = np.empty(24)
        ref.qs_step(0, e_ref)
    with lib_context() as ctx:
        load_mol(ctx, 0, m)
        ctx.set_wait_limits(*limits)
        with pytest.raises(MolgwError) as ei:
            ctx.rpa(0, np.empty(95))            # host output: synchronises
        assert ei.value.code == code
        ctx.set_wait_limits()                   # defaults back
        ctx.sync()
        load_mol(ctx, 0, m)                     # the same state as the clean context
        e = np.empty(24)
        ctx.qs_step(0, e)
        ctx.sync()
    assert np.array_equal(e, e_ref)


def test_timeout_inside_a_large_panel_launch():
    """A barrier timeout in a panel launch of a 1,600-transition Casida matrix (a grid of
    many CTAs on every SM): every CTA leaves, the call reports MOLGW_E_TIMEOUT, and the
    same context then reproduces a clean run bit for bit."""
    from paper_2210_17093_gb300 import MolgwError
    m = sy.molecule(100, 20, 300, 5)
    nov = 20 * 80
    with lib_context() as ref:
        load_mol(ref, 0, m)
        om_ref = np.empty(nov)
        ref.rpa(0, om_ref)
    with lib_context() as ctx:
        load_mol(ctx, 0, m)
        ctx.set_wait_limits(0, -1)
        with pytest.raises(MolgwError) as ei:
            ctx.rpa(0, np.empty(nov))
        assert ei.value.code == E_TIMEOUT
        ctx.set_wait_limits()
        ctx.sync()
        load_mol(ctx, 0, m)
        om = np.empty(nov)
        ctx.rpa(0, om)
    assert np.array_equal(om, om_ref)


def test_wait_limits_need_a_context():
    from paper_2210_17093_gb300 import native
    assert native.load().molgw_b200_set_wait_limits(None, 0, 0) == E_ARG
