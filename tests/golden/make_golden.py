"""Writes the files of tests/golden/ from the CPU oracle only.

Workload: one closed-shell molecule, n_basis=24, n_occ=5, n_aux=72, seed 0,
eta = 1e-3 Ha.  qsgw_nb24_no5_na72_seed0.json: one RI-qsGW pass (Eqs. AO.to.MO,
Casida, w.residue, Sigma.c.GW, Sigma.c.qsGW.real, K, H, GEP of arXiv 2210.17093).
qsmp2_g0w0_nb24_no5_na72_seed0.json: one qsMP2 pass (Eqs. Sigma.c.MP2,
Sigma.c.qsMP2.real) and the one-shot G0W0 energies (diagonal of Eq. Sigma.c.GW,
linearised).  The values are the oracle's; the paper prints no worked example.

With the argument ``C`` it writes instead qsgw_nb400_no80_na1200_seed4.npz: one
RI-qsGW pass of the 400/80/1200 workload (25,600 transitions), seed 4, eta = 1e-3
Ha -- Omega_s, the updated energies eps', Sigma_x and the Hermitised Sigma_c
(upper triangles, both matrices are symmetric) and min D_t.  The residues are
formed one orbital at a time (``keep_w=False``): whole, w would take 33 GB.  It
takes about 15 minutes on 8 x86 cores and ~35 GB of host memory.
Run from the repository root:
    python tests/golden/make_golden.py          # the 24/5/72 files
    python tests/golden/make_golden.py C        # the 400/80/1200 file
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synthetic as sy  # noqa: E402
from oracle import qsgw  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "qsgw_nb24_no5_na72_seed0.json")
OUT2 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "qsmp2_g0w0_nb24_no5_na72_seed0.json")
OUT_C = os.path.join(os.path.dirname(os.path.abspath(__file__)), "qsgw_nb400_no80_na1200_seed4.npz")


def main_config_c():
    import time

    import numpy as np
    nb, no, na, seed = 400, 80, 1200, 4
    t0 = time.time()
    m = sy.molecule(nb, no, na, seed)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], no, sy.ETA, keep_w=False)
    iu = np.triu_indices(nb)
    np.savez_compressed(
        OUT_C,
        source=np.array("oracle/qsgw.py qsgw_pass(keep_w=False); equations of arXiv 2210.17093 Sec. II"),
        workload=np.array([nb, no, na, seed]),
        eta=np.array(sy.ETA),
        Omega=r["Omega"],
        eps_new=r["eps_new"],
        sigma_x_upper=r["sigma_x"][iu],
        sigma_c_upper=r["sigma_c"][iu],
        min_D=np.array(r["D"].min()),
        trace_M=np.array(np.trace(r["M"])),
    )
    print(f"wrote {OUT_C} in {time.time() - t0:.0f} s")


def main():
    m = sy.molecule(24, 5, 72, 0)
    r = qsgw.qsgw_pass(m["L"], m["eps"], m["C"], 5, sy.ETA)
    doc = {
        "source": "oracle/qsgw.py qsgw_pass; equations of arXiv 2210.17093 Sec. II",
        "workload": {"n_basis": 24, "n_occ": 5, "n_aux": 72, "seed": 0, "eta": sy.ETA},
        "Omega": r["Omega"].tolist(),
        "eps_new": r["eps_new"].tolist(),
        "sigma_x": r["sigma_x"].tolist(),
        "sigma_c": r["sigma_c"].tolist(),
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=0)
    q = qsgw.qsmp2_pass(m["L"], m["eps"], m["C"], 5, sy.ETA)
    g = qsgw.g0w0_pass(m["L"], m["eps"], m["C"], 5, sy.ETA)
    doc2 = {
        "source": "oracle/qsgw.py qsmp2_pass and g0w0_pass; arXiv 2210.17093 Sec. II.C-D",
        "workload": {"n_basis": 24, "n_occ": 5, "n_aux": 72, "seed": 0, "eta": sy.ETA},
        "qsmp2_sigma_c": q["sigma_c"].tolist(),
        "qsmp2_eps_new": q["eps_new"].tolist(),
        "g0w0_eps_qp": g["eps_qp"].tolist(),
        "g0w0_z": g["Z"].tolist(),
    }
    with open(OUT2, "w") as f:
        json.dump(doc2, f, indent=0)


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "C":
        main_config_c()
    else:
        main()
