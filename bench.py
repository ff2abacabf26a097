#!/usr/bin/env python
"""Seconds per qsGW iteration of the RI-qsGW hot path on GB300 (one JSON line).

A step is one qsGW iteration of one molecule -- stages (a) ri_mo_transform,
(b) rpa_build, (c) rpa_eigensolve, (d) gw_residues, (e) sigma_assembly and
(f) qs_update -- through the C ABI, on seeded synthetic inputs (synthetic.py)
that stand in for the paper's cc-pVTZ alkanes.  Default workload: n_basis=200,
n_occ=40, n_aux=600 (6,400 transitions, M is 6400^2 float64), seed 1, plain
float64 on the GPU.  Each step continues the self-consistency from the previous
one (the orbitals are updated in place).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload B|C|E|D]

--workload D times the 64-molecule ragged batch (n_basis ~ U{40..160}) as one
qs_step(-1) per step on concurrent lanes with graph replay.

Under torchrun each rank runs an independent molecule (seed + rank): the units
are independent, there is no data-path collective, scaling is weak.
--impl reference times the CPU float64 oracle (oracle/) on the host cores.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as sy  # noqa: E402

METRIC = "s per qsGW iteration; TFLOP/s vs peak; mixed vs FP64 GPU speedup at ≤1 meV QP error"
WORKLOADS = {
    "A": dict(nb=24, no=5, na=72, seed=0),
    "B": dict(nb=200, no=40, na=600, seed=1),
    "C": dict(nb=400, no=80, na=1200, seed=4),
    "E": dict(nb=600, no=120, na=1800, seed=7),
}
# float64 peak derived from unit counts and clock: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz
# (NVIDIA lists 1.25 TFLOP/s FP64 for this part; a register-only DFMA loop measured 1.20).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def measured_peaks() -> dict:
    """Copy bandwidth and BF16 GEMM peaks measured on this GPU model (MEASURED_PEAKS.json
    beside this file), else one earlier GB300 measurement (6.8 TB/s, 1.9 PFLOP/s)."""
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "kind": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "kind": "fallback"}
# DRAM bytes the tridiagonalisation panel kernel moves per algorithmic byte (the lower
# triangle of the trailing matrix once per column), from one ncu capture of the panel of
# columns 1280..1343 at n = 6400: 4.564 GB measured for 6.629 GB algorithmic.
PANEL_TRAFFIC_RATIO = 4.564 / 6.629


def panel_bytes(n):
    """Algorithmic DRAM bytes of one reduction of M: sum over columns of the lower triangle."""
    return sum(4.0 * (n - i - 1) ** 2 for i in range(n - 1))


def workload_flops(nb, no, na):
    """Useful float64 flops per qsGW iteration (one product = 2 flops).

    Keys are the library's kernel classes where one class does the work.
    """
    n = no * (nb - no)
    return {
        # residues w^s_pm over the pairs m <= p (w^s_pm = w^s_mp: nb (nb + 1) / 2 pairs of
        # n_aux x n_ov products), then S += (w g) w^T per m
        "sigma": 1.0 * nb * (nb + 1) * na * n + 2.0 * nb ** 3 * n,
        # Householder reduction of M: symmetric matrix-vector products (2n^3/3) in the
        # panel kernel, rank-2k trailing updates of the lower triangle (2n^3/3) in the GEMM
        "tridiag_panel": 2.0 / 3.0 * n ** 3 + 2.0 * 64 * n * n,
        "tridiag_syr2k": 2.0 / 3.0 * n ** 3,
        "backtransform": 4.0 * na * n * n,                          # Q^T Xv and R = Y^T Z_T
        "rpa_build": 1.0 * na * n * n,                              # lower half of Xv Xv^T
        "ri_mo_transform": 4.0 * na * nb ** 3,
        "sigma_x": 2.0 * nb * nb * na * no,
        "qs_update": 4.0 / 3.0 * nb ** 3 + 6.0 * nb ** 3,
    }


CLASSES = ["gemm_f64", "tridiag_panel", "tridiag_syr2k", "bisect", "twisted", "backtransform", "sigma",
           "gemm_tc", "misc"]
FLAG_TC_AB_BIT, FLAG_EIG_TC_BIT = 1 << 4, 1 << 5
# float64 instruction rate (2 per clock per SM), for the kernels counted in operations
FP64_PEAK_GOPS = 152 * 2 * 2.07e9 / 1e9
BISECT_ROUNDS = 7        # float64 rounds per eigenvalue after the float32 bracket (typical)


def pad64(k):
    return -(-k // 64) * 64


def stage_rooflines(nb, no, na, stages_ms, precision="fp64", flags=0):
    """Achieved fraction of its own roofline for every kernel class timed over one
    qsGW iteration: float64 classes against the float64 pipe (useful flops of
    workload_flops), tensor-core classes against the measured BF16 burst peak
    (executed digit products), the slicing kernel of (e) against the measured HBM
    copy bandwidth, and the bisection and twisted-vector kernels against the float64
    instruction rate (their operation counts are estimates, stated per class)."""
    n = no * (nb - no)
    f = workload_flops(nb, no, na)
    peaks = measured_peaks()
    fx = precision == "bf16x10"
    tc_ab = fx and bool(flags & FLAG_TC_AB_BIT)
    eig_tc = bool(flags & FLAG_EIG_TC_BIT)
    out = {}

    def put(k, work, unit, peak, bound, what, extra=None):
        ms = stages_ms.get(k)
        if not ms or ms <= 0:
            return
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        ach = work / (ms / 1e3) / scale
        d = {"ms": round(ms, 3), "bound": bound, "work": what, "achieved": round(ach, 4), "peak": round(peak, 4),
             "unit": unit, "frac": round(ach / peak, 4)}
        if extra:
            d.update(extra)
        out[k] = d

    bf16 = peaks["bf16_tflops"]
    panel = f["tridiag_panel"] + 2.0 / 3.0 * nb ** 3
    if eig_tc:
        # the integer mat-vec reads the 8-byte image of the lower triangle of A22 once per
        # column (n^3/6 elements) and builds it once per 64-column panel (read float64,
        # write the image: 16 B per element of the lower triangle, n^3/384 elements)
        ms = stages_ms.get("tridiag_panel")
        put("tridiag_panel", 8.0 * n ** 3 / 6.0 + 16.0 * n ** 3 / 384.0, "GB/s", peaks["hbm_gbs"], "hbm",
            "integer mat-vec: 8-byte tile images of A22's lower triangle read once per column, built once per panel",
            {"fp64_equivalent_tflops": round(panel / (ms / 1e3) / 1e12, 3) if ms else None})
    else:
        put("tridiag_panel", panel, "TFLOP/s", FP64_PEAK_TFLOPS, "alu",
            "2n^3/3 + 128n^2 (symmetric mat-vecs, column updates) for M and H")
    syr2k = f["tridiag_syr2k"] + 2.0 / 3.0 * nb ** 3
    bt = f["backtransform"] + 2.0 * nb ** 3
    if eig_tc:
        for k, useful in (("tridiag_syr2k", syr2k), ("backtransform", bt)):
            ms = stages_ms.get(k)
            put(k, 28.0 * useful, "TFLOP/s", bf16, "tensor",
                "28 BF16 digit products per useful float64 multiply-add (7-digit fixed point)",
                {"fp64_equivalent_tflops": round(useful / (ms / 1e3) / 1e12, 3) if ms else None})
    else:
        put("tridiag_syr2k", syr2k, "TFLOP/s", FP64_PEAK_TFLOPS, "alu", "2n^3/3 rank-2k updates of the lower triangle")
        put("backtransform", bt, "TFLOP/s", FP64_PEAK_TFLOPS, "alu", "4 n_aux n^2 (Q^T Xv, R = Y^T Z_T) + C' = C U")
    put("bisect", 4.0 * BISECT_ROUNDS * 5.0 * (n * n + nb * nb) / 1e0, "Gop/s", FP64_PEAK_GOPS, "alu",
        f"estimated: 4 lanes x {BISECT_ROUNDS} float64 rounds x 5 operations per Sturm step, n steps per eigenvalue")
    put("twisted", 12.0 * (n * n + nb * nb), "Gop/s", FP64_PEAK_GOPS, "alu (serial recurrences: latency)",
        "estimated: 3 passes x 4 float64 operations per step, n steps per eigenvector")
    if fx:
        groups = -(-pad64(na) // 1024)
        nbytes = nb * nb * n * (8 * groups + 2 * 4 * 2)
        put("sigma", nbytes, "GB/s", peaks["hbm_gbs"], "hbm",
            "k_fx_sigma_slices: w partials read (8 B per 1024-wide group), digits of w and g w written (2 x 4 x 2 B)")
        ex = 10.0 * 2 * (nb * nb * n * pad64(na) + nb * nb * nb * pad64(n))
        if tc_ab:
            ex += 10.0 * 2 * (2 * na * nb * nb * pad64(nb) + 0.5 * n * n * pad64(na))
        put("gemm_tc", ex, "TFLOP/s", bf16, "tensor",
            "10 BF16 digit products per useful multiply-add: (d), (e)" + (", (a), (b)" if tc_ab else ""))
    else:
        put("sigma", f["sigma"], "TFLOP/s", FP64_PEAK_TFLOPS, "alu",
            "residues over the pairs m <= p and the Sigma_c contraction, float64")
    g64 = f["sigma_x"] + 2.0 * nb * nb * na + 6.0 * nb ** 3
    if not tc_ab:
        g64 += f["ri_mo_transform"] + f["rpa_build"]
    put("gemm_f64", g64, "TFLOP/s", FP64_PEAK_TFLOPS, "alu",
        ("" if tc_ab else "(a) 4 n_aux nb^3, (b) n_aux n^2, ") + "Sigma_x, J, the H and h_MO rotations")
    return out


def config_dict(wl, precision):
    nb, no, na = wl["nb"], wl["no"], wl["na"]
    n = no * (nb - no)
    return {
        "workload": f"closed-shell RI-qsGW iteration, n_basis={nb}, n_occ={no}, n_aux={na}, "
                    f"{n} transitions, seed {wl['seed']} (+rank)",
        "n_basis": nb, "n_occ": no, "n_aux": na, "n_transitions": n, "eta_ha": sy.ETA,
        "precision": precision,
        "l2": f"inputs larger than L2: L {na * nb * nb * 8 / 1e6:.0f} MB, M {n * n * 8 / 1e6:.0f} MB per step",
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.seek(0)
        return summarise_clocks(self.f.read())


def summarise_clocks(text):
    """Median SM clock, maximum SM clock and the throttle reasons seen in the CSV rows of
    ClockSampler.Q (noheader, nounits); rows that do not parse are skipped."""
    rows = [r for r in csv.reader(io.StringIO(text)) if len(r) >= 9]
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        try:
            sm.append(float(r[1]))
            smax = float(r[2])
        except ValueError:
            continue
        for k, nm in enumerate(names):
            if r[5 + k].strip().lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
            "reasons": sorted(reasons), "samples": len(sm)}


def molecule_seed(wl, rank):
    """Weak scaling: rank r runs its own molecule of the workload's shape, seed + r."""
    return wl["seed"] + rank


def batch_seeds(rank):
    """Weak scaling of the batch: rank r runs 64 molecules of its own, seeds 100..163 + 64 r."""
    return [s + 64 * rank for s in sy.BATCH_SEEDS]


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except ImportError:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_steps(wl, steps, warmup, eta):
    """Time `steps` oracle iterations after `warmup` (the CPU float64 reference)."""
    from oracle import qsgw
    m = sy.molecule(wl["nb"], wl["no"], wl["na"], wl["seed"])
    L, eps, C, h = m["L"], m["eps"], m["C"], None
    for _ in range(warmup):
        r = qsgw.qsgw_pass(L, eps, C, wl["no"], eta, h)
        eps, C, h = r["eps_new"], r["C_new"], r["h_mo_new"]
    t0 = time.perf_counter()
    for _ in range(steps):
        r = qsgw.qsgw_pass(L, eps, C, wl["no"], eta, h)
        eps, C, h = r["eps_new"], r["C_new"], r["h_mo_new"]
    return (time.perf_counter() - t0) / max(steps, 1)


# CPU seconds of one oracle iteration per workload on 16 Neoverse-V2 cores (measured), and
# the CPU time the reference arm allows itself
ORACLE_S_PER_ITER = {"A": 0.05, "B": 9.3, "C": 420.0, "E": 2400.0}
ORACLE_BUDGET_S = 240.0


def oracle_step_counts(wl, steps, warmup):
    """Steps and warm-up of the oracle arm: those requested when they fit the CPU budget,
    else as many steps as fit after one warm-up (at least one)."""
    key = next((k for k, v in WORKLOADS.items() if v == wl), "B")
    t = ORACLE_S_PER_ITER.get(key, 10.0)
    if (steps + warmup) * t <= ORACLE_BUDGET_S:
        return steps, warmup
    w = min(warmup, 1)
    return max(1, min(steps, int(ORACLE_BUDGET_S / t) - w)), w


def run_reference(args, wl):
    world, rank, local, dist = dist_setup()
    if rank != 0:
        return 0
    steps, warmup = oracle_step_counts(wl, args.steps, args.warmup)
    t = oracle_steps(wl, steps, warmup, sy.ETA)
    cores = os.cpu_count()
    sample = (f"{steps} oracle iteration(s) after {warmup} warm-up of the same workload "
              f"(seed {wl['seed']}), NumPy float64 with multithreaded BLAS"
              + ("" if (steps, warmup) == (args.steps, args.warmup) else
                 f"; {args.steps} steps after {args.warmup} requested, cut to keep the CPU run near 4 minutes"))
    line = {
        "impl": "reference", "metric": METRIC, "value": t, "unit": "s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warmup, "ms_per_step": t * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(wl, "fp64"),
        "cpu_baseline": {"value": t, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": t, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_reference_batch(args):
    """The oracle on workload D: each step one oracle iteration of a bounded sample of
    8 of the 64 molecules, scaled to the whole batch (rank 0 only)."""
    world, rank, local, dist = dist_setup()
    if rank != 0:
        return 0
    from oracle import qsgw
    mols = [sy.batch_molecule(s) for s in batch_seeds(0)]
    sample = mols[:8]
    steps, warmup = min(args.steps, 3), min(args.warmup, 1)
    for _ in range(warmup):
        qsgw.qsgw_pass(sample[0]["L"], sample[0]["eps"], sample[0]["C"], sample[0]["n_occ"], sy.ETA)
    t0 = time.perf_counter()
    for _ in range(steps):
        for m in sample:
            qsgw.qsgw_pass(m["L"], m["eps"], m["C"], m["n_occ"], sy.ETA)
    t = (time.perf_counter() - t0) / steps * len(mols) / len(sample)
    desc = (f"one oracle iteration of molecules {sy.BATCH_SEEDS[0]}..{sy.BATCH_SEEDS[7]} (n_basis "
            f"{', '.join(str(m['n_basis']) for m in sample)}) per step, time x {len(mols)}/{len(sample)}")
    line = {
        "impl": "reference", "metric": METRIC, "value": t, "unit": "s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warmup, "ms_per_step": t * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "ragged batch of 64 closed-shell RI-qsGW iterations (oracle sample)",
                   "molecules": len(mols), "eta_ha": sy.ETA},
        "cpu_baseline": {"value": t, "unit": "s", "cores": os.cpu_count(), "kind": "oracle", "sample": desc},
        "e2e": {"value": t, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


GOLDEN_C = os.path.join(ROOT, "tests", "golden", "qsgw_nb400_no80_na1200_seed4.npz")
HA_MEV = 27211.386


def one_pass(m, precision, flags, local, st, fetch_b=False):
    """One qsGW iteration of molecule m from its input orbitals through the C ABI, every
    kernel class event-timed on the context stream.  Returns the pass time, the time
    per class, and the pass's Omega, Sigma_x, Sigma_c and updated energies (and B on
    the device when fetch_b).  Buffers are allocated inside the first pass (a few tens
    of ms at these sizes, inside the time)."""
    import torch
    from paper_2210_17093_gb300 import Context
    nb, no, na = m["n_basis"], m["n_occ"], m["n_aux"]
    n = no * (nb - no)
    dev = f"cuda:{local}"
    out = {}
    with Context(precision=precision, device=local, eta=sy.ETA, stream=st, flags=flags) as ctx:
        L_d = torch.from_numpy(m["L"]).to(dev)
        ctx.set_ri(0, nb, na, L_d)
        ctx.set_orbitals(0, no, torch.from_numpy(m["eps"]).to(dev), torch.from_numpy(m["C"]).to(dev))
        ctx.sync()
        del L_d
        torch.cuda.empty_cache()
        ctx.set_timing(CLASSES)
        ctx.kernel_stats(reset=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        ctx.qs_step(0)
        e1.record(st)
        torch.cuda.synchronize()
        out["s"] = e0.elapsed_time(e1) / 1e3
        stats = ctx.kernel_stats(reset=True)
        out["stages_ms"] = {k: round(v[1], 2) for k, v in stats.items() if v[0]}
        om, sx, sc, ep = np.empty(n), np.empty(nb * nb), np.empty(nb * nb), np.empty(nb)
        ctx.fetch(0, "Omega", om)
        ctx.fetch(0, "sigma_x", sx)
        ctx.fetch(0, "sigma_c", sc)
        ctx.fetch(0, "eps", ep)
        out.update(Omega=om, sigma_x=sx.reshape(nb, nb), sigma_c=sc.reshape(nb, nb), eps_new=ep)
        if fetch_b:
            B = torch.empty(na * nb * nb, dtype=torch.float64, device=dev)
            ctx.fetch(0, "B", B)
            out["B"] = B
    return out


def vs_golden(r, g):
    """Errors of one pass against the oracle's stored values (upper triangles of Sigma)."""
    nb = r["eps_new"].shape[0]
    iu = np.triu_indices(nb)
    rel = lambda a, b: float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    d_eps = float(np.max(np.abs(r["eps_new"] - g["eps_new"])))
    return {"omega_max_abs_ha": float(np.max(np.abs(r["Omega"] - g["Omega"]))),
            "qp_max_abs_ha": d_eps, "qp_max_abs_meV": d_eps * HA_MEV,
            "sigma_x_rel": rel(r["sigma_x"][iu], g["sigma_x_upper"]),
            "sigma_c_rel": rel(r["sigma_c"][iu], g["sigma_c_upper"])}


def config_c_line(local, st):
    """Workload 400/80/1200 (25,600 transitions), seed 4: one float64 pass and two
    BF16X10 passes (TC_AB; and TC_AB + EIG_TC), each against the oracle's stored values."""
    wl = WORKLOADS["C"]
    m = sy.molecule(wl["nb"], wl["no"], wl["na"], wl["seed"])
    g = dict(np.load(GOLDEN_C)) if os.path.exists(GOLDEN_C) else None
    out = {"workload": "n_basis=400, n_occ=80, n_aux=1200, 25600 transitions, seed 4, one pass from the "
                       "input orbitals (M 5.2 GB)",
           "oracle_values": "tests/golden/qsgw_nb400_no80_na1200_seed4.npz (written by the CPU oracle)"
           if g is not None else None}
    runs = (("fp64", "fp64", 0), ("mixed", "bf16x10", FLAG_TC_AB_BIT),
            ("mixed_eig_tc", "bf16x10", FLAG_TC_AB_BIT | FLAG_EIG_TC_BIT))
    t64 = None
    for name, prec, flags in runs:
        r = one_pass(m, prec, flags, local, st)
        d = {"s_per_pass": round(r["s"], 3), "precision": prec, "flags": flags, "stages_ms": r["stages_ms"],
             "roofline_stages": stage_rooflines(wl["nb"], wl["no"], wl["na"], r["stages_ms"], prec, flags)}
        if t64 is None:
            t64 = r["s"]
        else:
            d["speedup_vs_fp64"] = round(t64 / r["s"], 3)
        if g is not None:
            d["vs_oracle"] = vs_golden(r, g)
            bar = 1e-8 if prec == "fp64" else 1.0 / HA_MEV
            d["meets_bar"] = bool(d["vs_oracle"]["qp_max_abs_ha"] <= bar and d["vs_oracle"]["omega_max_abs_ha"] <= bar
                                  and d["vs_oracle"]["sigma_c_rel"] <= 1e-6 and d["vs_oracle"]["sigma_x_rel"] <= 1e-6)
        out[name] = d
    return out


def config_e_line(local, st):
    """Workload 600/120/1800 (57,600 transitions, M 26.5 GB), seed 7: one BF16X10 pass
    (TC_AB + EIG_TC) with per-stage times and fractions, and checks that hold at any size."""
    import torch
    wl = WORKLOADS["E"]
    nb, no, na = wl["nb"], wl["no"], wl["na"]
    m = sy.molecule(nb, no, na, wl["seed"])
    flags = FLAG_TC_AB_BIT | FLAG_EIG_TC_BIT
    r = one_pass(m, "bf16x10", flags, local, st, fetch_b=True)
    n = no * (nb - no)
    eps = torch.from_numpy(m["eps"]).to(r["B"].device)
    D = (eps[no:][None, :] - eps[:no][:, None]).reshape(-1)            # t = i nv + (a - no)
    Bia = r["B"].view(na, nb, nb)[:, :no, no:].reshape(na, n)
    tr_m = float((D * D).sum() + 4.0 * (D * (Bia * Bia).sum(0)).sum())
    del Bia, r["B"]
    torch.cuda.empty_cache()
    om = r["Omega"]
    sum_om2 = float(np.sum(om * om))
    return {"workload": "n_basis=600, n_occ=120, n_aux=1800, 57600 transitions (M 26.5 GB), seed 7, one pass "
                        "from the input orbitals; BF16X10 with TC_AB and EIG_TC",
            "s_per_pass": round(r["s"], 3), "stages_ms": r["stages_ms"],
            "roofline_stages": stage_rooflines(nb, no, na, r["stages_ms"], "bf16x10", flags),
            "checks": {"sum_omega2_vs_trace_M_rel": abs(sum_om2 - tr_m) / tr_m,
                       "omega_min": float(om.min()), "min_D": float(D.min().item()),
                       "omega_min_ge_min_D": bool(om.min() >= float(D.min().item())),
                       "sigma_x_asym": float(np.max(np.abs(r["sigma_x"] - r["sigma_x"].T))),
                       "sigma_c_asym": float(np.max(np.abs(r["sigma_c"] - r["sigma_c"].T))),
                       "finite": bool(np.all(np.isfinite(om)) and np.all(np.isfinite(r["eps_new"])))}}


def run_ours(args, wl):
    import torch

    world, rank, local, dist = dist_setup()
    from paper_2210_17093_gb300 import FLAG_EIG_TC, FLAG_QSMP2, FLAG_TC_AB, Context

    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    nb, no, na = wl["nb"], wl["no"], wl["na"]
    n = no * (nb - no)
    m = sy.molecule(nb, no, na, molecule_seed(wl, rank))
    st = torch.cuda.Stream(device=dev)
    L_d = torch.from_numpy(m["L"]).to(dev)
    eps_d = torch.from_numpy(m["eps"]).to(dev)
    C_d = torch.from_numpy(m["C"]).to(dev)
    torch.cuda.synchronize()
    flops = workload_flops(nb, no, na)
    total_flops = sum(flops.values())

    with Context(precision=args.precision, device=local, eta=sy.ETA, stream=st) as ctx:
        ctx.set_ri(0, nb, na, L_d)
        ctx.set_orbitals(0, no, eps_d, C_d)
        ctx.autotune()               # setup: tile sides per GEMM shape; the orbitals put back
        for _ in range(args.warmup):
            ctx.qs_step(0)
        ctx.sync()
        dominant = args.dominant
        ctx.set_timing([dominant])
        ctx.kernel_stats(reset=True)
        l0 = ctx.launch_count()
        sampler = ClockSampler(local)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier(dist)
        torch.cuda.synchronize()
        sampler.start()
        e0.record(st)
        for _ in range(args.steps):
            ctx.qs_step(0)
        e1.record(st)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        barrier(dist)
        launches = ctx.launch_count() - l0
        t_dev = e0.elapsed_time(e1) / 1e3
        kstats = ctx.kernel_stats(reset=True)
        ctx.set_timing([])
        t_max = max_over_ranks(dist, t_dev)

        # per-class breakdown: one more iteration with every class event-timed
        ctx.set_timing(["gemm_f64", "tridiag_panel", "tridiag_syr2k", "bisect", "twisted",
                        "backtransform", "sigma", "gemm_tc", "misc"])
        ctx.kernel_stats(reset=True)
        ctx.qs_step(0)
        breakdown = ctx.kernel_stats(reset=True)
        ctx.set_timing([])

        # end to end through the public API: pinned host inputs and outputs every step
        L_h = torch.from_numpy(m["L"]).pin_memory()
        eps_h = torch.from_numpy(m["eps"]).pin_memory()
        C_h = torch.from_numpy(m["C"]).pin_memory()
        eps_o = torch.empty(nb, dtype=torch.float64).pin_memory()
        C_o = torch.empty(nb * nb, dtype=torch.float64).pin_memory()
        for _ in range(1):
            ctx.set_ri(0, nb, na, L_h)
            ctx.set_orbitals(0, no, eps_h, C_h)
            ctx.qs_step(0, eps_o, C_o)
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 3))
        for _ in range(e2e_steps):
            ctx.set_ri(0, nb, na, L_h)
            ctx.set_orbitals(0, no, eps_h, C_h)
            ctx.qs_step(0, eps_o, C_o)
        torch.cuda.synchronize()
        t_e2e = (time.perf_counter() - t0) / e2e_steps
        barrier(dist)
        t_e2e = max_over_ranks(dist, t_e2e)
        eps_fp64_step1 = eps_o.numpy().copy()     # float64 step from the input orbitals

    def variant(precision: str, flags: int, stages: str) -> dict:
        """Another precision / flag set on the same molecule: time per step, and its
        first step against the float64 GPU path (which matches the oracle to 1e-8 Ha)."""
        with Context(precision=precision, device=local, eta=sy.ETA, stream=st, flags=flags) as mctx:
            mctx.set_ri(0, nb, na, L_d)
            mctx.set_orbitals(0, no, eps_d, C_d)
            mctx.autotune()
            e1 = torch.empty(nb, dtype=torch.float64).pin_memory()
            mctx.qs_step(0, e1)
            for _ in range(max(0, args.warmup - 1)):
                mctx.qs_step(0)
            mctx.sync()
            m0 = torch.cuda.Event(enable_timing=True)
            m1 = torch.cuda.Event(enable_timing=True)
            barrier(dist)
            torch.cuda.synchronize()
            m0.record(st)
            for _ in range(args.steps):
                mctx.qs_step(0)
            m1.record(st)
            torch.cuda.synchronize()
            t_v = max_over_ranks(dist, m0.elapsed_time(m1) / 1e3)
            mctx.set_timing(["gemm_f64", "tridiag_panel", "tridiag_syr2k", "bisect", "twisted",
                             "backtransform", "sigma", "gemm_tc", "misc"])
            mctx.kernel_stats(reset=True)
            mctx.qs_step(0)
            vbreak = mctx.kernel_stats(reset=True)
        err = float(np.max(np.abs(e1.numpy() - eps_fp64_step1)))
        out = {"precision": precision, "flags": flags, "stages": stages,
               "ms_per_step": t_v / args.steps * 1e3,
               "speedup_vs_fp64": (t_max / args.steps) / (t_v / args.steps),
               "qp_error_vs_fp64_meV": err * 27211.386,
               "meets_1meV": bool(err * 27211.386 <= 1.0),
               "stages_ms": {k: round(v[1], 3) for k, v in vbreak.items() if v[0]},
               "roofline_stages": stage_rooflines(nb, no, na, {k: v[1] for k, v in vbreak.items() if v[0]},
                                                  precision, flags)}
        tc_ms = vbreak.get("gemm_tc", (0, 0.0))[1]
        sg_ms = vbreak.get("sigma", (0, 0.0))[1]
        if precision == "bf16x10" and sg_ms > 0:
            # the fused denominator kernel of (e): per (p, m, s) it reads w (float64, one
            # partial per 1024-wide group of n_aux) and writes w and g*w as 4 BF16 digits each
            peaks = measured_peaks()
            groups = -(-(-(-na // 64) * 64) // 1024)
            nbytes = nb * nb * n * (8 * groups + 2 * 4 * 2)
            out["sigma_assembly"] = {
                "kernel": "k_fx_sigma_slices (float64 eps_p - eps_m -/+ Omega_s, g, digits of w and g w)",
                "bytes": nbytes, "ms": sg_ms, "achieved_gbs": nbytes / (sg_ms / 1e3) / 1e9,
                "frac_of_hbm": nbytes / (sg_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                "peak_gbs": peaks["hbm_gbs"], "peak_kind": peaks["kind"],
                "note": "bound by the float64 pipe (~15 float64 operations per element), not by HBM"}
        if precision == "bf16x10" and tc_ms > 0:
            # ten BF16 digit products per useful multiply-add: w = B_m^T R (K = n_aux padded
            # to 64) and S = (g w) w^T (K = n_basis x n_ov padded to 64)
            peaks = measured_peaks()
            pad = lambda k: -(-k // 64) * 64
            ex_flops = 10 * 2 * (nb * nb * n * pad(na) + nb * nb * nb * pad(n))
            if flags & FLAG_TC_AB:
                # (a): two GEMMs M = n_aux n_basis, N = n_basis, K = n_basis padded; (b): lower
                # 64-blocks of Xv Xv^T (about half of n_ov^2 n_aux padded)
                ex_flops += 10 * 2 * (2 * na * nb * nb * pad(nb) + 0.5 * n * n * pad(na))
            out["tensor"] = {"kernels": "gemm_tc class: fx_gemm_kernel<4> of (d)+(e)"
                                        + (" and (a), (b)" if flags & FLAG_TC_AB else ""),
                             "executed_tflops": ex_flops / (tc_ms / 1e3) / 1e12,
                             "frac_of_bf16_peak": ex_flops / (tc_ms / 1e3) / 1e12 / peaks["bf16_tflops"],
                             "peak_tflops": peaks["bf16_tflops"], "peak_kind": peaks["kind"] + " bf16 burst"}
        return out

    def qsmp2_variant(precision: str, flags: int, ref_eps=None) -> dict:
        """qsMP2 (MOLGW_FLAG_QSMP2) iterations on the same molecule: no RPA."""
        with Context(precision=precision, device=local, eta=sy.ETA, stream=st, flags=FLAG_QSMP2 | flags) as q:
            q.set_ri(0, nb, na, L_d)
            q.set_orbitals(0, no, eps_d, C_d)
            q.autotune()
            e1 = torch.empty(nb, dtype=torch.float64).pin_memory()
            q.qs_step(0, e1)
            for _ in range(max(0, args.warmup - 1)):
                q.qs_step(0)
            q.sync()
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            barrier(dist)
            torch.cuda.synchronize()
            q0.record(st)
            for _ in range(args.steps):
                q.qs_step(0)
            q1.record(st)
            torch.cuda.synchronize()
            t_q = max_over_ranks(dist, q0.elapsed_time(q1) / 1e3) / args.steps
            q.set_timing(["gemm_f64", "sigma", "gemm_tc", "misc"])
            q.kernel_stats(reset=True)
            q.qs_step(0)
            qbreak = q.kernel_stats(reset=True)
        # useful flops: (p m|i a) and the exchange partner per summed orbital m, the
        # contraction S += [g (2A - X)] A^T, plus (a), Sigma_x and (f)
        f_sig = 2.0 * (2.0 * nb * nb * na * n) + 2.0 * nb ** 3 * n
        f_all = f_sig + flops["ri_mo_transform"] + flops["sigma_x"] + flops["qs_update"]
        out = {"precision": precision, "flags": FLAG_QSMP2 | flags,
               "method": "qsMP2: Eqs. (Sigma.c.MP2), (Sigma.c.qsMP2.real); (a), residues, (f)",
               "ms_per_step": t_q * 1e3, "tflops_useful": f_all / t_q / 1e12,
               "speedup_vs_qsgw_fp64": (t_max / args.steps) / t_q,
               "stages_ms": {k: round(v[1], 3) for k, v in qbreak.items() if v[0] and v[1] > 0},
               "eps_step1": e1.numpy().copy()}
        if precision == "fp64":
            sig_ms = qbreak.get("sigma", (0, 0.0))[1]
            out["roofline"] = {"kernel": "sigma class (gemm_f64 residues and contraction, k_apply_g_mp2)",
                               "bound": "alu", "achieved": (f_sig / (sig_ms / 1e3) / 1e12) if sig_ms > 0 else None,
                               "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                               "frac": (f_sig / (sig_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS) if sig_ms > 0 else None}
        else:
            tc_ms = qbreak.get("gemm_tc", (0, 0.0))[1]
            peaks = measured_peaks()
            pad = lambda k: -(-k // 64) * 64
            ex_flops = 10 * 2 * (2 * nb * nb * n * pad(na) + nb * nb * nb * pad(n))
            if flags & FLAG_TC_AB:
                ex_flops += 10 * 2 * (2 * na * nb * nb * pad(nb))
            out["tensor"] = {"kernels": "gemm_tc class: fx_gemm_kernel<4> (direct factor, exchange partner, "
                                        "Sigma contraction" + (", (a)" if flags & FLAG_TC_AB else "") + ")",
                             "executed_tflops": ex_flops / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None,
                             "frac_of_bf16_peak": ex_flops / (tc_ms / 1e3) / 1e12 / peaks["bf16_tflops"]
                             if tc_ms > 0 else None,
                             "peak_tflops": peaks["bf16_tflops"], "peak_kind": peaks["kind"] + " bf16 burst"}
        if ref_eps is not None:
            err = float(np.max(np.abs(out["eps_step1"] - ref_eps)))
            out["qp_error_vs_qsmp2_fp64_meV"] = err * 27211.386
            out["qp_error_relative"] = err / float(np.max(np.abs(ref_eps)))
            out["qp_max_abs_ha"] = float(np.max(np.abs(ref_eps)))
        return out

    def qsmp2_lines() -> dict:
        q64 = qsmp2_variant("fp64", 0)
        qfx = qsmp2_variant("bf16x10", FLAG_TC_AB, q64["eps_step1"])
        qfx["speedup_vs_qsmp2_fp64"] = q64["ms_per_step"] / qfx["ms_per_step"]
        q64.pop("eps_step1")
        qfx.pop("eps_step1")
        if world == 1 and not args.no_cpu_baseline:
            from oracle import qsgw
            mo = sy.molecule(nb, no, na, molecule_seed(wl, rank))
            t0 = time.perf_counter()
            qsgw.qsmp2_pass(mo["L"], mo["eps"], mo["C"], no, sy.ETA)
            q64["cpu_baseline"] = {"value": time.perf_counter() - t0, "unit": "s", "cores": os.cpu_count(),
                                   "kind": "oracle", "sample": "1 oracle qsMP2 iteration of the same molecule"}
        return {"fp64": q64, "mixed": qfx}

    def g0w0_lines() -> dict:
        """One-shot G0W0 (molgw_b200_g0w0_window) from the input orbitals, all states and the
        four frontier states.  Calls after the first reuse (a)-(c) of the unchanged
        orbitals, so the times are the G0W0 part: residues, diagonal sums, update."""
        out = {}
        with Context(precision="fp64", device=local, eta=sy.ETA, stream=st) as g:
            g.set_ri(0, nb, na, L_d)
            g.set_orbitals(0, no, eps_d, C_d)
            g.autotune()
            e_all = np.empty(nb)
            for name, lo, hi in (("all_states", 0, nb), ("window_4_frontier", no - 2, no + 2)):
                for _ in range(2):                      # warm-up
                    g.g0w0_window(0, lo, hi, np.empty(hi - lo))
                g0 = torch.cuda.Event(enable_timing=True)
                g1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                g0.record(st)
                for _ in range(args.steps):
                    g.g0w0_window(0, lo, hi)            # results stay on the device
                g1.record(st)
                torch.cuda.synchronize()
                out[name] = {"states": hi - lo, "ms_per_call_reusing_rpa": g0.elapsed_time(g1) / args.steps}
            g.fetch(0, "eps_qp", e_all)
        out["note"] = ("G0W0 after the first call reuses (a)-(c) of the current orbitals: the times are the "
                       "residues, the diagonal sums and the linearised update; (a)-(c) cost what they cost "
                       "in the qsGW iteration (stages_ms)")
        out["homo_lumo_qp_ha"] = [float(e_all[no - 1]), float(e_all[no])]
        return out

    def open_shell_line() -> dict:
        """One open-shell qsGW iteration on the same RI factors: n_occ up = n_occ, down =
        n_occ - 1 (the spin-down orbitals a rotation of the spin-up ones), float64."""
        rng = np.random.default_rng(7)
        Cdn, _ = np.linalg.qr(m["C"] + 0.3 * rng.standard_normal((nb, nb)))
        edn = np.sort(m["eps"] + 0.2 * rng.standard_normal(nb))
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        n_open = no * (nb - no) + (no - 1) * (nb - no + 1)
        with Context(precision="fp64", device=local, eta=sy.ETA, stream=st) as o:
            o.set_ri(0, nb, na, L_d)
            o.set_orbitals_open(0, no, no - 1, eps_d, d(edn), C_d, d(Cdn))
            o.autotune()
            o.qs_step(0)
            o.sync()
            t0e = torch.cuda.Event(enable_timing=True)
            t1e = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0e.record(st)
            steps = max(1, min(args.steps, 2))
            for _ in range(steps):
                o.qs_step(0)
            t1e.record(st)
            torch.cuda.synchronize()
            t = t0e.elapsed_time(t1e) / steps
        return {"method": "open-shell qsGW, float64: one RPA over the transitions of both spins",
                "n_occ_up_down": [no, no - 1], "n_transitions": n_open, "ms_per_step": t}

    extras = {}
    if world == 1 and not args.no_extra_configs:
        for key, fn in (("config_C", lambda: config_c_line(local, st)), ("config_E", lambda: config_e_line(local, st))):
            try:
                extras[key] = fn()
            except Exception as exc:          # a failed extra workload must not hide the main line
                extras[key] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()
        try:
            import copy
            bargs = copy.copy(args)
            bargs.steps, bargs.warmup, bargs.no_cpu_baseline = 3, 3, True
            bargs.dominant = "tridiag_panel"
            extras["batch_D"] = run_batch(bargs, setup=(world, rank, local, dist), emit=False)
        except Exception as exc:
            extras["batch_D"] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.empty_cache()
    qsmp2 = None if args.no_mp2 else qsmp2_lines()
    g0w0 = None if args.no_variants else g0w0_lines()
    open_shell = None if args.no_variants else open_shell_line()
    mixed = mixed_eig = fp64_eig = None
    if not args.no_mixed:
        ab = FLAG_TC_AB if args.mixed == "bf16x10" else 0
        mixed = variant(args.mixed, ab, "(a), (b), (d) and the Sigma contraction of (e) on tcgen05 tensor cores; "
                                        "eigensolvers (c), (f) and the denominators float64")
        mixed_eig = variant(args.mixed, ab | FLAG_EIG_TC,
                            "as 'mixed', and the eigensolvers' SYR2K and back-transformation GEMMs on 7-digit "
                            "fixed point (tensor cores) and the panel mat-vecs on 53-bit integer images (integer "
                            "multiply-adds), both float64-accurate normwise; bisection and twisted vectors float64")
        fp64_eig = variant("fp64", FLAG_EIG_TC,
                           "float64, with the eigensolvers' SYR2K and back-transformation GEMMs on 7-digit "
                           "fixed point (tensor cores) and the panel mat-vecs on 53-bit integer images "
                           "(float64 accuracy normwise)")

    if rank != 0:
        return 0
    value = t_max / (args.steps * world)
    nl, kms = kstats[dominant]
    dom_flops = flops.get(dominant)
    achieved = dom_flops * args.steps / (kms / 1e3) / 1e12 if (dom_flops and kms > 0) else None
    traffic = None
    if dominant == "tridiag_panel" and nl:
        # measured bytes per algorithmic byte x algorithmic bytes, per launch (all panel launches)
        traffic = PANEL_TRAFFIC_RATIO * panel_bytes(n) * args.steps / nl
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else args.precision,
        "data": "synthetic", "config": config_dict(wl, args.precision),
        "tflops": total_flops / (t_max / args.steps) / 1e12,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": {
            "kernel": dominant, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
            "traffic": traffic, "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
            "traffic_source": "ncu dram__bytes_read+write of one panel launch (n=6400, columns 1280-1343: "
                              "4.56 GB for 6.63 GB algorithmic, part of the trailing matrix served by L2), "
                              "that ratio times the algorithmic bytes per launch",
            "launches": nl, "event_ms": kms,
        },
        "stages_ms": {k: round(v[1], 3) for k, v in breakdown.items() if v[0]},
        "roofline_stages": stage_rooflines(nb, no, na, {k: v[1] for k, v in breakdown.items() if v[0]},
                                           args.precision, 0),
        "mixed": mixed,
        "mixed_eig_tc": mixed_eig,
        "fp64_eig_tc": fp64_eig,
        "qsmp2": qsmp2,
        "g0w0": g0w0,
        "open_shell": open_shell,
        "e2e": {"value": t_e2e, "unit": "s",
                "h2d_bytes_per_step": int((na * nb * nb + nb + nb * nb) * 8),
                "d2h_bytes_per_step": int((nb + nb * nb) * 8)},
    }
    line["config"]["autotuned"] = "float64 GEMM tile sides (molgw_b200_autotune, during setup)"
    if world == 1 and not args.no_cpu_baseline:
        t_cpu = oracle_steps(wl, 1, 0, sy.ETA)
        line["cpu_baseline"] = {
            "value": t_cpu, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 oracle iteration of the same workload (seed {wl['seed']}), NumPy float64, "
                      f"BLAS threads = host cores"}
    line.update(extras)
    line["headline"] = headline(line)
    print(json.dumps(line, separators=(",", ":")))
    return 0


def headline(line):
    """The figures of the line in a few hundred characters, last on the line so that a
    reader of its tail sees them: s per iteration per path and workload, speed-ups,
    errors against the oracle, per-stage roofline fractions."""
    r3 = lambda x: None if x is None else float(f"{x:.4g}")
    h = {"B_fp64_s": r3(line["value"]), "B_panel_frac": r3(line["roofline"]["frac"])}
    for k in ("mixed", "mixed_eig_tc", "fp64_eig_tc"):
        v = line.get(k)
        if v:
            h[f"B_{k}_s"] = r3(v["ms_per_step"] / 1e3)
            h[f"B_{k}_x"] = r3(v["speedup_vs_fp64"])
            h[f"B_{k}_qp_meV"] = r3(v["qp_error_vs_fp64_meV"])
    h["B_stage_frac"] = {k: r3(v["frac"]) for k, v in line.get("roofline_stages", {}).items()}
    c = line.get("config_C") or {}
    for k in ("fp64", "mixed", "mixed_eig_tc"):
        v = c.get(k)
        if isinstance(v, dict):
            h[f"C_{k}_s"] = r3(v["s_per_pass"])
            if "speedup_vs_fp64" in v:
                h[f"C_{k}_x"] = r3(v["speedup_vs_fp64"])
            if "vs_oracle" in v:
                h[f"C_{k}_qp_meV"] = r3(v["vs_oracle"]["qp_max_abs_meV"])
                h[f"C_{k}_ok"] = v["meets_bar"]
    if "error" in c:
        h["C_error"] = c["error"][:80]
    e = line.get("config_E") or {}
    if "s_per_pass" in e:
        h["E_s"] = r3(e["s_per_pass"])
        h["E_stage_frac"] = {k: r3(v["frac"]) for k, v in e["roofline_stages"].items()}
        h["E_checks_ok"] = bool(e["checks"]["omega_min_ge_min_D"] and e["checks"]["finite"]
                                and e["checks"]["sum_omega2_vs_trace_M_rel"] < 1e-6)
    elif "error" in e:
        h["E_error"] = e["error"][:80]
    d = line.get("batch_D") or {}
    if "value" in d:
        h["D_s"] = r3(d["value"])
        h["D_launches_per_step"] = int(d["gpu_launches"] / max(d["steps"], 1))
    elif "error" in d:
        h["D_error"] = d["error"][:80]
    return h


def run_batch(args, setup=None, emit=True):
    """Workload D: 64 molecules (n_basis ~ U{40..160}, seeds 100-163 + 64 x rank) as one
    qs_step(-1) per step on concurrent lanes, replayed from a captured graph.  With
    emit=False the line is returned instead of printed (setup: the caller's
    (world, rank, local, dist))."""
    import torch

    world, rank, local, dist = setup if setup is not None else dist_setup()
    from paper_2210_17093_gb300 import FLAG_EIG_TC, FLAG_GRAPH, FLAG_TC_AB, Context

    torch.cuda.set_device(local)
    seeds = batch_seeds(rank)
    mols = [sy.batch_molecule(s) for s in seeds]
    st = torch.cuda.Stream(device=f"cuda:{local}")
    flops = {}
    for m in mols:
        for k, v in workload_flops(m["n_basis"], m["n_occ"], m["n_aux"]).items():
            flops[k] = flops.get(k, 0.0) + v
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    host = [(pin(m["L"]), pin(m["eps"]), pin(m["C"])) for m in mols]
    prec = args.batch_precision
    flags = FLAG_GRAPH | (FLAG_TC_AB if prec != "fp64" else 0) | (0 if args.batch_no_eig_tc else FLAG_EIG_TC)
    with Context(precision=prec, device=local, eta=sy.ETA, stream=st, max_mols=len(mols),
                 flags=flags, lanes=0) as ctx:
        def load():
            for k, (m, (L, e, C)) in enumerate(zip(mols, host)):
                ctx.set_ri(k, m["n_basis"], m["n_aux"], L)
                ctx.set_orbitals(k, m["n_occ"], e, C)
        load()
        ctx.sync()
        tuned_lanes = ctx.autotune()      # setup: trial steps, the orbitals put back after each
        dominant = args.dominant
        # graph replays record no kernel events: the roofline comes from the first
        # (directly issued) warm-up step, whose panel launches are those of every step
        ctx.set_timing([dominant])
        ctx.kernel_stats(reset=True)
        ctx.qs_step(-1)
        kstats = ctx.kernel_stats(reset=True)
        ctx.set_timing([])
        for _ in range(args.warmup - 1):
            ctx.qs_step(-1)
        ctx.sync()
        l0 = ctx.launch_count()
        r0 = ctx.graph_replays()
        sampler = ClockSampler(local)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier(dist)
        torch.cuda.synchronize()
        sampler.start()
        e0.record(st)
        for _ in range(args.steps):
            ctx.qs_step(-1)
        e1.record(st)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        t_max = max_over_ranks(dist, e0.elapsed_time(e1) / 1e3)
        launches = ctx.launch_count() - l0
        replays = ctx.graph_replays() - r0
        # end to end: inputs from pinned host memory, qs_step(-1), eps of every molecule to the host
        outs = [torch.empty(m["n_basis"], dtype=torch.float64).pin_memory() for m in mols]
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        load()
        ctx.qs_step(-1)
        for k, o in enumerate(outs):
            ctx.fetch(k, "eps", o)
        t_e2e = max_over_ranks(dist, time.perf_counter() - t0)
    if rank != 0:
        return 0 if emit else None
    nl, kms = kstats[dominant]
    dom_flops = flops.get(dominant)
    achieved = dom_flops / (kms / 1e3) / 1e12 if (dom_flops and kms > 0) else None
    roofline = {"kernel": dominant, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                "traffic": None, "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"}
    if dominant == "tridiag_panel" and flags & FLAG_EIG_TC and kms > 0:
        # the integer mat-vec (every lane): the 8-byte tile images read once per column and
        # built once per panel, as in the single-molecule stage rooflines
        nov = [m["n_occ"] * (m["n_basis"] - m["n_occ"]) for m in mols]
        nbytes = sum(8.0 * n ** 3 / 6.0 + 16.0 * n ** 3 / 384.0 for n in nov)
        hbm = measured_peaks()["hbm_gbs"]
        ach = nbytes / (kms / 1e3) / 1e9
        roofline = {"kernel": dominant, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)",
                    "work": "integer mat-vec: 8-byte tile images of each Casida matrix's lower triangle read once "
                            "per column, built once per panel",
                    "fp64_equivalent_tflops": achieved}
    roofline.update({"launches": nl, "event_ms": kms,
                     "note": "one directly issued step (graph replays record no events); launches of "
                             "concurrent lanes overlap, so achieved = work / summed launch time"})
    nbs = [m["n_basis"] for m in mols]
    line = {
        "metric": METRIC, "value": t_max / (args.steps * world), "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else prec, "data": "synthetic",
        "config": {"workload": f"ragged batch of {len(mols)} closed-shell RI-qsGW iterations, n_basis "
                               f"{min(nbs)}..{max(nbs)} (U{{40..160}}), n_occ = round(n_basis/5), n_aux = 3 n_basis, "
                               f"seeds {seeds[0]}..{seeds[-1]}; one qs_step(-1) per step on autotuned lanes, "
                               f"graph replay", "molecules": len(mols), "precision": prec,
                   "stages_on_tensor_cores": ("(a), (b), (d), (e)" if prec != "fp64" else "none")
                   + ("; the eigensolvers' SYR2K and back-transformation GEMMs on 7-digit fixed point "
                      "and their panel mat-vecs on 53-bit integer images (float64 accuracy normwise)"
                      if flags & FLAG_EIG_TC else ""), "eta_ha": sy.ETA,
                   "l2": "inputs larger than L2 (RI factors and Casida matrices of 64 molecules, ~10 GB)"},
        "tflops": sum(flops.values()) / (t_max / args.steps) / 1e12,
        "gpu_launches": int(launches), "graph_replays": int(replays), "autotuned_lanes": tuned_lanes,
        "clocks": clocks,
        "roofline": roofline,
        "e2e": {"value": t_e2e, "unit": "s",
                "h2d_bytes_per_step": int(sum((m["n_aux"] * m["n_basis"] ** 2 + m["n_basis"] + m["n_basis"] ** 2) * 8
                                              for m in mols)),
                "d2h_bytes_per_step": int(sum(m["n_basis"] * 8 for m in mols))},
    }
    if world == 1 and not args.no_cpu_baseline:
        # a bounded sample: 4 molecules of the batch, one oracle iteration each, scaled to 64
        from oracle import qsgw
        sample = mols[:4]
        t0 = time.perf_counter()
        for m in sample:
            qsgw.qsgw_pass(m["L"], m["eps"], m["C"], m["n_occ"], sy.ETA)
        t_cpu = (time.perf_counter() - t0) * len(mols) / len(sample)
        line["cpu_baseline"] = {
            "value": t_cpu, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"one oracle iteration of molecules {seeds[0]}..{seeds[3]} (n_basis "
                      f"{', '.join(str(m['n_basis']) for m in sample)}), time x {len(mols)}/{len(sample)}"}
    if not emit:
        return line
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["D"], default="B",
                    help="B/C/E: one molecule; D: the 64-molecule ragged batch")
    ap.add_argument("--batch-precision", choices=["fp64", "bf16x3", "tf32x3", "bf16x6", "bf16x10"],
                    default="bf16x10", help="precision of workload D")
    ap.add_argument("--precision", choices=["fp64", "bf16x3", "tf32x3", "bf16x6", "bf16x10"], default="fp64")
    ap.add_argument("--dominant", default="tridiag_panel", help="kernel class reported in 'roofline'")
    ap.add_argument("--mixed", choices=["bf16x3", "tf32x3", "bf16x6", "bf16x10"], default="bf16x10",
                    help="precision of the split-precision path reported under 'mixed'")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-mp2", action="store_true", help="skip the qsMP2 line item")
    ap.add_argument("--no-variants", action="store_true", help="skip the G0W0 and open-shell line items")
    ap.add_argument("--batch-no-eig-tc", action="store_true",
                    help="workload D: keep the eigensolvers' trailing updates in float64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="skip the 400/80/1200 and 600/120/1800 passes and the batch object (N=1 only)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.workload == "D":
        if args.impl == "reference":
            return run_reference_batch(args)
        return run_batch(args)
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
