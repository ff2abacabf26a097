"""Seeded synthetic inputs for one closed-shell RI-qsGW pass.

This module only draws inputs; it holds none of the method's arithmetic, so both
the CPU oracle (``oracle/``) and the CUDA path can take their inputs from it.

What is drawn (closed shell, real orbitals, orthonormal AO basis so S = I):

* occupied energies  eps_i ~ U[-20, -0.3] Ha (sorted), virtual energies
  eps_a ~ U[0.05, 5] Ha (sorted) -- the MO energies of Eq. (GEP);
* MO coefficients C (Eq. MO): a random orthogonal n_basis x n_basis matrix from
  the QR factorisation of a Gaussian matrix, column signs fixed by diag(R) > 0;
* three-centre RI factors (P|mu nu) (the paper names RI in Sec. II.B but prints
  no RI equation; the factors are read as already contracted with the metric, so
  (mu nu|la ta) = sum_P (P|mu nu)(P|la ta), which is positive semidefinite):
  G_P ~ N(0,1) symmetrised as (G + G^T)/sqrt(2), mixed by a lower-bidiagonal
  L with L_00 = s_0, L_PP = s_P sqrt(1 - rho^2), L_P,P-1 = s_P rho, rho = 0.5,
  s_P = 0.5 exp(-P/24), so that each (P|mu nu) is N(0, s_P^2) off the diagonal.

Draw order for one molecule with ``rng = numpy.random.default_rng(seed)``:
eps_occ, eps_virt, the Gaussian matrix for C, then G.  A batch molecule first
draws its basis size n_basis = rng.integers(40, 161) from its own seed, then
n_occ = round(n_basis / 5) and n_aux = 3 n_basis.

The paper's workloads are cc-pVTZ alkanes C1..C7 (86..434 basis functions,
Sec. III); their integrals are not available, so these inputs stand in for them
with the sizes below.
"""
from __future__ import annotations

import numpy as np

RHO = 0.5
SIGMA0 = 0.5
SIGMA_DECAY = 24.0

# name -> (n_basis, n_occ, n_aux, seeds)
CONFIGS = {
    "A": (24, 5, 72, (0,)),
    "B": (200, 40, 600, (1, 2, 3)),
    "C": (400, 80, 1200, (4, 5, 6)),
    "E": (600, 120, 1800, (7,)),
}
BATCH_SEEDS = tuple(range(100, 164))
ETA = 1e-3


def aux_sigma(n_aux: int) -> np.ndarray:
    """Per-function standard deviation s_P = 0.5 exp(-P/24), P 0-based."""
    return SIGMA0 * np.exp(-np.arange(n_aux, dtype=np.float64) / SIGMA_DECAY)


def _draw(rng: np.random.Generator, n_basis: int, n_occ: int, n_aux: int) -> dict:
    if not (0 < n_occ < n_basis) or n_aux < 1:
        raise ValueError("need 0 < n_occ < n_basis and n_aux >= 1")
    n_virt = n_basis - n_occ
    eps_occ = np.sort(rng.uniform(-20.0, -0.3, n_occ))
    eps_virt = np.sort(rng.uniform(0.05, 5.0, n_virt))
    eps = np.concatenate([eps_occ, eps_virt])
    q, r = np.linalg.qr(rng.standard_normal((n_basis, n_basis)))
    C = q * np.sign(np.diag(r))[None, :]
    s = aux_sigma(n_aux)
    L = np.empty((n_aux, n_basis, n_basis), dtype=np.float64)
    prev = None
    for P in range(n_aux):
        g = rng.standard_normal((n_basis, n_basis))
        g = (g + g.T) / np.sqrt(2.0)
        if P == 0:
            L[P] = s[0] * g
        else:
            L[P] = s[P] * np.sqrt(1.0 - RHO * RHO) * g + s[P] * RHO * prev
        prev = g
    return {
        "n_basis": n_basis,
        "n_occ": n_occ,
        "n_aux": n_aux,
        "eps": np.ascontiguousarray(eps),
        "C": np.ascontiguousarray(C),
        "L": L,
    }


def molecule(n_basis: int, n_occ: int, n_aux: int, seed: int) -> dict:
    """One molecule of the given sizes; see the module docstring for the recipe."""
    rng = np.random.default_rng(seed)
    mol = _draw(rng, n_basis, n_occ, n_aux)
    mol["seed"] = seed
    return mol


def batch_molecule(seed: int) -> dict:
    """One molecule of the ragged batch: n_basis ~ U{40..160} drawn first."""
    rng = np.random.default_rng(seed)
    n_basis = int(rng.integers(40, 161))
    n_occ = int(round(n_basis / 5))
    mol = _draw(rng, n_basis, n_occ, 3 * n_basis)
    mol["seed"] = seed
    return mol


def config_molecules(name: str, seeds=None) -> list:
    """The molecules of a named workload ("A", "B", "C", "E" or "D" = batch)."""
    if name == "D":
        return [batch_molecule(s) for s in (seeds or BATCH_SEEDS)]
    nb, no, na, default_seeds = CONFIGS[name]
    return [molecule(nb, no, na, s) for s in (seeds or default_seeds)]


def scale_ri(mol: dict, lam: float) -> dict:
    """Copy of ``mol`` with the RI factors multiplied by ``lam`` (coupling strength)."""
    out = dict(mol)
    out["L"] = mol["L"] * lam
    return out
