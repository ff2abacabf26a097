"""Shared helpers of the GPU tests: build/load the library, run the oracle, compare."""
import numpy as np
import pytest


def lib_context(**kw):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_17093_gb300 import Context
    # run on torch's current stream so that device outputs are ordered before
    # any later torch read of them
    kw.setdefault("stream", torch.cuda.current_stream())
    return Context(**kw)


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def rel_max(a, b):
    """max |a - b| / max |b| (the Sigma tolerance measure)."""
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def load_mol(ctx, mol, m, device=True, h_core=None):
    nb, na, no = m["n_basis"], m["n_aux"], m["n_occ"]
    put = to_dev if device else np.ascontiguousarray
    ctx.set_ri(mol, nb, na, put(m["L"]))
    ctx.set_orbitals(mol, no, put(m["eps"]), put(m["C"]), None if h_core is None else put(h_core))
