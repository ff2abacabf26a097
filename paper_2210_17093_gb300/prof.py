"""Small drivers to profile the library's kernels (e.g. under ncu).

    python -m paper_2210_17093_gb300.prof eigh N [REPS [FLAGS [MATVEC]]]
        float64 symmetric eigensolve of a random N x N matrix (tridiagonalisation,
        bisection, twisted vectors, full back-transformation) through molgw_b200_eigh
        (FLAGS: e.g. 32 for MOLGW_FLAG_EIG_TC; MATVEC: the panel kernel's mat-vec
        under it, auto, fp64, tc or int);
    python -m paper_2210_17093_gb300.prof qsgw NB NO NA PRECISION [REPS [FLAGS [MATVEC]]]
        qsGW iterations of one synthetic molecule (seed 1) at the given precision
        (FLAGS: extra MOLGW_FLAG_* bits, e.g. 32 for MOLGW_FLAG_EIG_TC);
    python -m paper_2210_17093_gb300.prof batch PRECISION LANES [REPS]
        qsGW iterations of the 64-molecule ragged batch (n_basis ~ U{40..160},
        seeds 100-163) as one mol = -1 call on LANES concurrent streams;
    python -m paper_2210_17093_gb300.prof trace NB NO NA PRECISION FLAGS SEED
        one qsGW pass of one synthetic molecule, timed per stage, with checks that
        hold at any size: sum_s Omega_s^2 = tr M = sum_t D_t^2 + 4 sum_t D_t sum_P (B^P_t)^2
        (from the library's own B, in float64 on the host), Omega_min >= min D_t, and
        Sigma_x, Sigma_c symmetric.

Each prints the per-kernel-class event times of every repetition.
"""
from __future__ import annotations

import os
import sys
import time


def _stats(ctx):
    return {k: round(v[1], 2) for k, v in ctx.kernel_stats(reset=True).items() if v[0]}


def eigh(n: int, reps: int = 1, flags: int = 0, matvec: str = "auto") -> None:
    import torch

    from . import Context, FLAG_KTIMING
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g)
    A = (A + A.T).contiguous()
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    Z = torch.empty(n * n, dtype=torch.float64, device="cuda")
    with Context(stream=torch.cuda.current_stream(), flags=FLAG_KTIMING | flags) as ctx:
        ctx.set_panel_matvec(matvec)
        for r in range(reps):
            ctx.kernel_stats(reset=True)
            torch.cuda.synchronize()
            t = time.perf_counter()
            ctx.eigh(A, w, Z)
            torch.cuda.synchronize()
            print(f"eigh n={n} rep {r}: {(time.perf_counter() - t) * 1e3:.1f} ms", _stats(ctx), flush=True)


def qsgw(nb: int, no: int, na: int, precision: str, reps: int = 2, flags: int = 0) -> None:
    import numpy as np
    import torch

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synthetic as sy

    from . import Context, FLAG_KTIMING
    m = sy.molecule(nb, no, na, 1)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with Context(precision=precision, stream=torch.cuda.current_stream(), flags=FLAG_KTIMING | flags,
                 eta=sy.ETA) as ctx:
        ctx.set_ri(0, nb, na, d(m["L"]))
        ctx.set_orbitals(0, no, d(m["eps"]), d(m["C"]))
        for r in range(reps):
            ctx.kernel_stats(reset=True)
            torch.cuda.synchronize()
            t = time.perf_counter()
            ctx.qs_step(0)
            ctx.sync()
            print(f"qs_step nb={nb} {precision} flags={flags} rep {r}: {(time.perf_counter() - t) * 1e3:.1f} ms", _stats(ctx),
                  flush=True)


def batch(precision: str, lanes: int, reps: int = 2) -> None:
    import numpy as np

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synthetic as sy

    from . import Context, FLAG_KTIMING
    mols = sy.config_molecules("D")
    with Context(precision=precision, max_mols=len(mols), flags=FLAG_KTIMING, eta=sy.ETA, lanes=lanes) as ctx:
        for k, m in enumerate(mols):
            ctx.set_ri(k, m["n_basis"], m["n_aux"], np.ascontiguousarray(m["L"]))
            ctx.set_orbitals(k, m["n_occ"], np.ascontiguousarray(m["eps"]), np.ascontiguousarray(m["C"]))
        ctx.sync()
        for r in range(reps):
            ctx.kernel_stats(reset=True)
            t = time.perf_counter()
            ctx.qs_step(-1)
            ctx.sync()
            print(f"batch {precision} lanes={lanes} rep {r}: {(time.perf_counter() - t) * 1e3:.1f} ms", _stats(ctx),
                  flush=True)


def trace(nb: int, no: int, na: int, precision: str, flags: int, seed: int) -> None:
    import numpy as np
    import torch

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synthetic as sy

    from . import Context, FLAG_KTIMING
    t0 = time.perf_counter()
    m = sy.molecule(nb, no, na, seed)
    print(f"inputs drawn in {time.perf_counter() - t0:.1f} s", flush=True)
    nv = nb - no
    nov = no * nv
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with Context(precision=precision, stream=torch.cuda.current_stream(), flags=FLAG_KTIMING | flags,
                 eta=sy.ETA) as ctx:
        ctx.set_ri(0, nb, na, d(m["L"]))
        ctx.set_orbitals(0, no, d(m["eps"]), d(m["C"]))
        del m["L"]
        ctx.sync()
        ctx.kernel_stats(reset=True)
        t = time.perf_counter()
        om = np.empty(nov)
        ctx.rpa(0, om)
        print(f"rpa (a)-(c): {time.perf_counter() - t:.2f} s", _stats(ctx), flush=True)
        t = time.perf_counter()
        sx = np.empty((nb, nb))
        sc = np.empty((nb, nb))
        ctx.sigma(0, sx, sc)
        print(f"sigma (d)-(e): {time.perf_counter() - t:.2f} s", _stats(ctx), flush=True)
        t = time.perf_counter()
        eps = np.empty(nb)
        ctx.qs_step(0, eps)
        print(f"qs_update (f): {time.perf_counter() - t:.2f} s", _stats(ctx), flush=True)
        B = np.empty(na * nb * nb)
        ctx.fetch(0, "B", B)
    B = B.reshape(na, nb, nb)
    e = m["eps"]
    D = (e[None, no:] - e[:no, None]).reshape(-1)                 # t = i nv + a'
    k2 = np.einsum("Pia,Pia->ia", B[:, :no, no:], B[:, :no, no:]).reshape(-1)
    trM = float(np.sum(D * D) + 4.0 * np.sum(D * k2))
    s2 = float(np.sum(om * om))
    print(f"sum Omega^2 = {s2:.12e}  tr M = {trM:.12e}  rel diff = {abs(s2 - trM) / trM:.2e}")
    print(f"Omega_min = {om.min():.10f} >= min D = {D.min():.10f}: {bool(om.min() >= D.min() * (1 - 1e-12))}")
    print(f"Sigma_x asym = {np.max(np.abs(sx - sx.T)):.1e}  Sigma_c asym = {np.max(np.abs(sc - sc.T)):.1e}  "
          f"max|Sigma_c| = {np.max(np.abs(sc)):.3e}  QP eps range [{eps.min():.6f}, {eps.max():.6f}]", flush=True)


if __name__ == "__main__":
    a = sys.argv[1:]
    if a and a[0] == "eigh":
        eigh(int(a[1]), int(a[2]) if len(a) > 2 else 1, int(a[3]) if len(a) > 3 else 0, a[4] if len(a) > 4 else "auto")
    elif a and a[0] == "batch":
        batch(a[1], int(a[2]), int(a[3]) if len(a) > 3 else 2)
    elif a and a[0] == "trace":
        trace(int(a[1]), int(a[2]), int(a[3]), a[4], int(a[5]), int(a[6]))
    elif a and a[0] == "qsgw":
        qsgw(int(a[1]), int(a[2]), int(a[3]), a[4], int(a[5]) if len(a) > 5 else 2, int(a[6]) if len(a) > 6 else 0)
    else:
        print(__doc__)
        sys.exit(2)
