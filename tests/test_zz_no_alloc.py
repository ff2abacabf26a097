"""molgw_b200_eigh_noalloc against molgw_b200_eigh, through the C ABI.

The allocation-free entry point serves callers that cannot allocate device
memory when they need the decomposition (a pool allocator that owns all device
memory, a latency-bound loop that cannot pay for cudaMalloc/cudaFree).  It must
give the results of the allocating entry point on consecutive calls that share
its one static workspace.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _sym(n, seed, spread):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(10.0 ** rng.uniform(0, spread, n)) * rng.choice([-1.0, 1.0], n)
    A = (Q * lam[None, :]) @ Q.T
    return 0.5 * (A + A.T)


def test_noalloc_matches_eigh_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_17093_gb300 import Context, native

    lib = native.load()
    st = torch.cuda.current_stream()
    cases = [(200, 1, 4.0), (77, 2, 2.0), (256, 3, 1.0)]   # different sizes back to back
    with Context(stream=st) as ctx:
        for n, seed, spread in cases:
            A = _sym(n, seed, spread)
            Ad = torch.from_numpy(A).cuda()
            w = torch.empty(n, dtype=torch.float64, device="cuda")
            Z = torch.empty(n * n, dtype=torch.float64, device="cuda")
            rc = lib.molgw_b200_eigh_noalloc(n, ctypes.c_void_p(Ad.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                             ctypes.c_void_p(Z.data_ptr()), ctypes.c_void_p(st.cuda_stream))
            assert rc == 0, native.STATUS.get(rc, rc)
            w_ref = np.empty(n)
            Z_ref = np.empty((n, n))
            ctx.eigh(np.ascontiguousarray(A), w_ref, Z_ref)
            w_na, Z_na = w.cpu().numpy(), Z.cpu().numpy().reshape(n, n)
            scale = np.abs(w_ref).max()
            # the tolerance of the eigensolver tests
            assert np.max(np.abs(w_na - w_ref)) <= 1e-12 * scale * n ** 0.5
            assert np.max(np.abs(Z_na - Z_ref)) <= 1e-10
            assert np.max(np.abs(A @ Z_na - Z_na * w_na[None, :])) <= 1e-11 * scale


def test_noalloc_eigenvalues_only_and_default_stream():
    """Z = NULL (eigenvalues only) and stream = NULL (the legacy default stream) give
    the eigenvalues of molgw_b200_eigh, twice in a row."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_17093_gb300 import Context, native

    lib = native.load()
    with Context(stream=torch.cuda.current_stream()) as ctx:
        for n, seed, spread in [(130, 5, 3.0), (256, 6, 2.0)]:
            A = _sym(n, seed, spread)
            Ad = torch.from_numpy(A).cuda()
            w = torch.empty(n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            rc = lib.molgw_b200_eigh_noalloc(n, ctypes.c_void_p(Ad.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                             None, None)
            assert rc == 0, native.STATUS.get(rc, rc)
            w_ref = np.empty(n)
            ctx.eigh(np.ascontiguousarray(A), w_ref, None)
            assert np.max(np.abs(w.cpu().numpy() - w_ref)) <= 1e-12 * np.abs(w_ref).max() * n ** 0.5


def test_noalloc_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_17093_gb300 import native

    lib = native.load()
    n = native.NOALLOC_NMAX + 1
    A = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert lib.molgw_b200_eigh_noalloc(n, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                       None, None) == -1          # above the stated maximum
    h = np.zeros(4)
    assert lib.molgw_b200_eigh_noalloc(2, h.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(w.data_ptr()),
                                       None, None) == -1          # host input
    hp = torch.zeros(4, dtype=torch.float64).pin_memory()        # pinned host memory is host memory
    assert lib.molgw_b200_eigh_noalloc(2, ctypes.c_void_p(hp.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                       None, None) == -1
    assert lib.molgw_b200_eigh_noalloc(2, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(hp.data_ptr()),
                                       None, None) == -1          # host output
    assert lib.molgw_b200_eigh_noalloc(0, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                       None, None) == -1          # empty
