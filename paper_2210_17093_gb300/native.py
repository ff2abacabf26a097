"""ctypes binding of the RI-qsGW C ABI (include/molgw_gb300.h).

Argument marshalling only: every stage runs inside the CUDA library.  Arrays may
be torch tensors (CUDA or CPU) or NumPy arrays; they must be float64 and
C-contiguous.  The library must have been built (``paper_2210_17093_gb300.build``);
loading fails loudly otherwise -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmolgw_gb300.so")

PREC = {"fp64": 0, "bf16x3": 1, "tf32x3": 2, "bf16x6": 3, "bf16x10": 4}
FLAG_FULL_XPY = 1
FLAG_KTIMING = 2
FLAG_GRAPH = 4
FLAG_USE_STREAM = 8
FLAG_TC_AB = 16
FLAG_EIG_TC = 32
FLAG_QSMP2 = 64

ITEM = {"B": 0, "Omega": 1, "R": 2, "sigma_x": 3, "sigma_c": 4, "J": 5, "h_mo": 6, "eps": 7, "C": 8,
        "eps_qp": 9, "Z": 10, "sigma_c_diag": 11}
KERNELS = ["gemm_f64", "tridiag_panel", "tridiag_syr2k", "bisect", "twisted", "backtransform",
           "sigma", "gemm_tc", "misc"]

STATUS = {0: "MOLGW_OK", -1: "MOLGW_E_ARG", -2: "MOLGW_E_STATE", -3: "MOLGW_E_NOMEM",
          -4: "MOLGW_E_CUDA", -5: "MOLGW_E_NOCONV", -6: "MOLGW_E_TIMEOUT", -7: "MOLGW_E_NUMERIC"}

# Every symbol include/molgw_gb300.h declares.
EXPORTS = ["molgw_b200_create", "molgw_b200_set_ri", "molgw_b200_set_orbitals", "molgw_b200_rpa",
           "molgw_b200_sigma", "molgw_b200_qs_step", "molgw_b200_sync", "molgw_b200_fetch",
           "molgw_b200_rpa_matrix", "molgw_b200_eigh", "molgw_b200_kernel_stats",
           "molgw_b200_launch_count", "molgw_b200_set_timing", "molgw_b200_destroy",
           "molgw_b200_status_string", "molgw_b200_eigh_noalloc", "molgw_b200_graph_replays",
           "molgw_b200_tc_gemm", "molgw_b200_autotune", "molgw_b200_lanes", "molgw_b200_g0w0",
           "molgw_b200_g0w0_window", "molgw_b200_inject_fault", "molgw_b200_set_orbitals_open",
           "molgw_b200_plan_batch", "molgw_b200_set_wait_limits", "molgw_b200_set_panel_matvec"]
# mat-vec of the tridiagonalisation's panel kernel with FLAG_EIG_TC (molgw_matvec)
MATVEC = {"auto": 0, "fp64": 1, "tc": 2, "int": 3}
NOALLOC_NMAX = 256


class MolgwError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)} ({status_string(code)})")


class Opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("max_mols", ctypes.c_int32), ("device", ctypes.c_int32),
                ("eta", ctypes.c_double), ("stream", ctypes.c_void_p), ("flags", ctypes.c_uint32),
                ("lanes", ctypes.c_int32)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the shared library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run python -m paper_2210_17093_gb300.build)")
    lib = ctypes.CDLL(path)
    vp, ip, dp, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
    sig = {
        "molgw_b200_create": ([ctypes.POINTER(Opts), ctypes.POINTER(vp)], ip),
        "molgw_b200_set_ri": ([vp, ip, ip, ip, dp], ip),
        "molgw_b200_set_orbitals": ([vp, ip, ip, dp, dp, dp], ip),
        "molgw_b200_set_orbitals_open": ([vp, ip, ip, ip, dp, dp, dp, dp, dp], ip),
        "molgw_b200_rpa": ([vp, ip, dp, dp], ip),
        "molgw_b200_sigma": ([vp, ip, dp, dp], ip),
        "molgw_b200_qs_step": ([vp, ip, dp, dp], ip),
        "molgw_b200_g0w0": ([vp, ip, dp, dp, dp], ip),
        "molgw_b200_g0w0_window": ([vp, ip, ip, ip, dp, dp, dp], ip),
        "molgw_b200_sync": ([vp], ip),
        "molgw_b200_inject_fault": ([vp, ip], ip),
        "molgw_b200_set_wait_limits": ([vp, ctypes.c_longlong, ip], ip),
        "molgw_b200_set_panel_matvec": ([vp, ip], ip),
        "molgw_b200_fetch": ([vp, ip, ip, dp, sz], ip),
        "molgw_b200_rpa_matrix": ([vp, ip, dp], ip),
        "molgw_b200_eigh": ([vp, ip, dp, dp, dp], ip),
        "molgw_b200_kernel_stats": ([vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double), ip], ip),
        "molgw_b200_launch_count": ([vp], ctypes.c_int64),
        "molgw_b200_graph_replays": ([vp], ctypes.c_int64),
        "molgw_b200_autotune": ([vp, ctypes.POINTER(ctypes.c_int32)], ip),
        "molgw_b200_lanes": ([vp], ctypes.c_int32),
        "molgw_b200_tc_gemm": ([vp, ip, ip, ip, ip, vp, vp, vp], ip),
        "molgw_b200_set_timing": ([vp, ctypes.c_uint32], ip),
        "molgw_b200_destroy": ([vp], ip),
        "molgw_b200_status_string": ([ip], ctypes.c_char_p),
        "molgw_b200_eigh_noalloc": ([ip, dp, dp, dp, vp], ip),
        "molgw_b200_plan_batch": ([ip, vp, vp, vp, vp, ctypes.c_uint32, ip, vp, vp], ip),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().molgw_b200_status_string(code).decode()
    except Exception:  # noqa: BLE001 - only used to decorate an error message
        return "?"


def plan_batch(n_basis, n_aux, n_occ, n_occ_dn=None, flags: int = 0, lanes: int = 0):
    """Lane plan of a batch without a device (molgw_b200_plan_batch): returns
    (lane_of, slot), int32 arrays over the molecules.  ``n_occ_dn`` None = all closed
    shells, else per molecule with -1 for a closed shell."""
    cols = [np.ascontiguousarray(x, dtype=np.int32) for x in (n_basis, n_aux, n_occ)]
    n = cols[0].size
    if any(c.size != n for c in cols):
        raise ValueError("n_basis, n_aux and n_occ must have the same length")
    dn = None if n_occ_dn is None else np.ascontiguousarray(n_occ_dn, dtype=np.int32)
    if dn is not None and dn.size != n:
        raise ValueError("n_occ_dn must have one entry per molecule")
    lane_of, slot = np.empty(n, np.int32), np.empty(n, np.int32)
    r = load().molgw_b200_plan_batch(n, cols[0].ctypes.data, cols[1].ctypes.data, cols[2].ctypes.data,
                                     None if dn is None else dn.ctypes.data, flags, lanes,
                                     lane_of.ctypes.data, slot.ctypes.data)
    if r < 0:
        raise MolgwError(r, "plan_batch")
    return lane_of, slot


def _ptr(a, n: int | None = None):
    """Raw data pointer of a float64 C-contiguous torch tensor or NumPy array (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be float64 and C-contiguous")
        if n is not None and a.size != n:
            raise ValueError(f"array has {a.size} elements, expected {n}")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be float64 and contiguous")
        if n is not None and a.numel() != n:
            raise ValueError(f"tensor has {a.numel()} elements, expected {n}")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check(code: int, what: str):
    if code != 0:
        raise MolgwError(code, what)


class Context:
    """One library context (include/molgw_gb300.h, molgw_b200_create)."""

    def __init__(self, precision: str = "fp64", max_mols: int = 1, device: int = 0,
                 eta: float = 1e-3, stream=None, flags: int = 0, lanes: int = 0):
        self._lib = load()
        o = Opts()
        o.struct_size = ctypes.sizeof(Opts)
        o.precision = PREC[precision]
        o.max_mols = max_mols
        o.device = device
        o.eta = eta
        if stream is not None:
            # an explicit stream (a torch stream or a raw handle) is always used, even
            # the legacy default stream whose handle is 0
            stream = stream if isinstance(stream, int) else stream.cuda_stream
            flags |= FLAG_USE_STREAM
        o.stream = stream
        o.flags = flags
        o.lanes = lanes
        h = ctypes.c_void_p()
        _check(self._lib.molgw_b200_create(ctypes.byref(o), ctypes.byref(h)), "molgw_b200_create")
        self._h = h
        self.sizes = {}
        self.open_nov = {}    # open-shell molecules: transitions of both spins

    def _hh(self):
        if self._h is None:
            raise RuntimeError("context is closed")
        return self._h

    def set_ri(self, mol: int, n_basis: int, n_aux: int, L):
        _check(self._lib.molgw_b200_set_ri(self._hh(), mol, n_basis, n_aux,
                                           _ptr(L, n_aux * n_basis * n_basis)), "set_ri")
        self.sizes[mol] = [n_basis, n_aux, None]
        self.open_nov.pop(mol, None)

    def set_orbitals(self, mol: int, n_occ: int, eps, C, h_core=None):
        nb = self.sizes[mol][0] if mol in self.sizes else None
        nn = None if nb is None else nb * nb
        _check(self._lib.molgw_b200_set_orbitals(self._hh(), mol, n_occ, _ptr(eps, nb), _ptr(C, nn),
                                                 _ptr(h_core, nn)), "set_orbitals")
        self.sizes[mol][2] = n_occ
        self.open_nov.pop(mol, None)

    def set_orbitals_open(self, mol: int, n_occ_up: int, n_occ_dn: int, eps_up, eps_dn, C_up, C_dn,
                          h_core=None):
        """Open shell: one set of orbitals per spin (molgw_b200_set_orbitals_open).  Later
        per-orbital outputs are the spin-up block followed by the spin-down block."""
        nb = self.sizes[mol][0] if mol in self.sizes else None
        nn = None if nb is None else nb * nb
        _check(self._lib.molgw_b200_set_orbitals_open(self._hh(), mol, n_occ_up, n_occ_dn, _ptr(eps_up, nb),
                                                      _ptr(eps_dn, nb), _ptr(C_up, nn), _ptr(C_dn, nn),
                                                      _ptr(h_core, nn)), "set_orbitals_open")
        self.sizes[mol][2] = n_occ_up
        self.open_nov[mol] = n_occ_up * (nb - n_occ_up) + n_occ_dn * (nb - n_occ_dn)

    def n_ov(self, mol: int):
        if mol in self.open_nov:
            return self.open_nov[mol]
        nb, _, no = self.sizes.get(mol, (None, None, None))
        return None if no is None else no * (nb - no)

    def _spins(self, mol: int) -> int:
        return 2 if mol in self.open_nov else 1

    def rpa(self, mol: int, omega=None, xpy=None):
        n = self.n_ov(mol) if mol >= 0 else None
        _check(self._lib.molgw_b200_rpa(self._hh(), mol, _ptr(omega, n), _ptr(xpy, None if n is None else n * n)),
               "rpa")

    def sigma(self, mol: int, sigma_x=None, sigma_c=None):
        nn = self._spins(mol) * self.sizes[mol][0] ** 2 if mol in self.sizes else None
        _check(self._lib.molgw_b200_sigma(self._hh(), mol, _ptr(sigma_x, nn), _ptr(sigma_c, nn)), "sigma")

    def qs_step(self, mol: int, eps_out=None, C_out=None):
        nb = self.sizes[mol][0] if mol in self.sizes else None
        k = self._spins(mol)
        _check(self._lib.molgw_b200_qs_step(self._hh(), mol, _ptr(eps_out, None if nb is None else k * nb),
                                            _ptr(C_out, None if nb is None else k * nb * nb)), "qs_step")

    def g0w0(self, mol: int, eps_qp=None, z=None, sigma_c_diag=None):
        nb = self.sizes[mol][0] if mol in self.sizes else None
        _check(self._lib.molgw_b200_g0w0(self._hh(), mol, _ptr(eps_qp, nb), _ptr(z, nb), _ptr(sigma_c_diag, nb)),
               "g0w0")

    def g0w0_window(self, mol: int, p_begin: int, p_end: int, eps_qp=None, z=None, sigma_c_diag=None):
        n = p_end - p_begin
        _check(self._lib.molgw_b200_g0w0_window(self._hh(), mol, p_begin, p_end, _ptr(eps_qp, n), _ptr(z, n),
                                                _ptr(sigma_c_diag, n)), "g0w0_window")

    def sync(self):
        _check(self._lib.molgw_b200_sync(self._hh()), "sync")

    def inject_fault(self, code: int):
        """Latch a device-side error code (test hook; see molgw_b200_inject_fault)."""
        _check(self._lib.molgw_b200_inject_fault(self._hh(), code), "inject_fault")

    def set_wait_limits(self, grid_spins: int = -1, bisect_rounds: int = -1):
        """Lower the bounds of the device waits (test hook; see molgw_b200_set_wait_limits);
        negative values restore the defaults."""
        _check(self._lib.molgw_b200_set_wait_limits(self._hh(), grid_spins, bisect_rounds), "set_wait_limits")

    def set_panel_matvec(self, kind: str = "auto"):
        """Choose the panel kernel's mat-vec under FLAG_EIG_TC: "auto", "fp64", "tc" or "int"
        (see molgw_b200_set_panel_matvec)."""
        _check(self._lib.molgw_b200_set_panel_matvec(self._hh(), MATVEC[kind]), "set_panel_matvec")

    def fetch(self, mol: int, item: str, out):
        n = out.size if isinstance(out, np.ndarray) else out.numel()
        _check(self._lib.molgw_b200_fetch(self._hh(), mol, ITEM[item], _ptr(out), n), f"fetch {item}")

    def rpa_matrix(self, mol: int, out):
        n = self.n_ov(mol)
        _check(self._lib.molgw_b200_rpa_matrix(self._hh(), mol, _ptr(out, None if n is None else n * n)),
               "rpa_matrix")

    def eigh(self, A, w, Z=None):
        n = w.size if isinstance(w, np.ndarray) else w.numel()
        _check(self._lib.molgw_b200_eigh(self._hh(), n, _ptr(A, n * n), _ptr(w, n), _ptr(Z, None if Z is None else n * n)),
               "eigh")

    def kernel_stats(self, reset: bool = False) -> dict:
        k = len(KERNELS)
        launches = (ctypes.c_int64 * k)()
        ms = (ctypes.c_double * k)()
        _check(self._lib.molgw_b200_kernel_stats(self._hh(), launches, ms, int(reset)), "kernel_stats")
        return {name: (int(launches[i]), float(ms[i])) for i, name in enumerate(KERNELS)}

    def set_timing(self, classes):
        """Time the named kernel classes (see KERNELS) with CUDA events; [] turns timing off."""
        mask = 0
        for name in classes:
            mask |= 1 << KERNELS.index(name)
        _check(self._lib.molgw_b200_set_timing(self._hh(), mask), "set_timing")

    def launch_count(self) -> int:
        return int(self._lib.molgw_b200_launch_count(self._hh()))

    def tc_gemm(self, A, B, C, digits: int = 0):
        """C[M][N] = sum_k A[m][k] B[n][k] on a tensor-core engine: the context's split
        (digits=0) or the fixed-point engine with 4 or 7 digits."""
        M, K = A.shape
        N = B.shape[0]
        _check(self._lib.molgw_b200_tc_gemm(self._hh(), digits, M, N, K, _ptr(A, M * K), _ptr(B, N * K),
                                            _ptr(C, M * N)), "tc_gemm")

    def autotune(self) -> int:
        """Time one qs_step(-1) per lane count (state restored after each), keep the fastest."""
        out = ctypes.c_int32(0)
        _check(self._lib.molgw_b200_autotune(self._hh(), ctypes.byref(out)), "autotune")
        return int(out.value)

    def lanes(self) -> int:
        return int(self._lib.molgw_b200_lanes(self._hh()))

    def graph_replays(self) -> int:
        """qs_step calls served from a captured graph (-1: capture failed, graphs off)."""
        return int(self._lib.molgw_b200_graph_replays(self._hh()))

    def close(self):
        if self._h is not None:
            h, self._h = self._h, None
            _check(self._lib.molgw_b200_destroy(h), "destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None:
                self._lib.molgw_b200_destroy(self._h)
                self._h = None
        except Exception:  # noqa: BLE001
            pass
