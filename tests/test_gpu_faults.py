"""Failure detection without a GPU fault: device-detected error codes latched by the
test hook molgw_b200_inject_fault travel through the API the way a bounded wait that
ran out would (returned by the next synchronising call, then cleared), and the
context stays usable."""
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
