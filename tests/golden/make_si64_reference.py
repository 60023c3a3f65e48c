"""Writes si64_reference.json: reference values of the 64-atom diamond Si cell (2x2x2
conventional cells, a = 10.26 bohr, seeded 0.05-bohr jitter, sp basis, S/H cut at 10 bohr,
L on 12 bohr) computed by the CPU oracle and, for the dense limit, by scipy.

The paper prints no worked example for this path (no energies, residuals or counts), so
the stored values are regression values of the oracle's own definitions: pattern block
counts (minimum-image pairs d^2 < R^2 plus self pairs), the Hotelling residuals
||S T - I||_F of ten steps from T_0 = I/sigma, the Palser-Manolopoulos start and twenty LNV
steps at N_e = 256, and the dense-limit band energy 2 sum_occ eps of the generalised
eigenproblem H c = eps S c.  Every value comes from oracle/ or scipy, never from the CUDA
path.  Run from the repository root: python tests/golden/make_si64_reference.py
"""
import json
import os
import sys

import numpy as np
import scipy.linalg as sl

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2205_08941_gb300 import inputs as I  # noqa: E402

RECIPE = {"ncell": 2, "a_bohr": 10.26, "sigma_bohr": 0.05, "seed": 1, "norb": 4,
          "r_S": 10.0, "r_L": 12.0, "n_electrons": 256.0, "hotelling_steps": 10,
          "lnv_steps": 20}


def compute():
    r = RECIPE
    cell = I.diamond_cell(r["ncell"], a=r["a_bohr"], sigma=r["sigma_bohr"], seed=r["seed"],
                          norb=r["norb"])
    Spb, Hpb = I.overlap_hamiltonian(cell, I.silicon_model(r["r_S"]))
    rS, rL = r["r_S"], r["r_L"]
    pats = {R: O.Pattern.of_cell(cell, R) for R in (rS, rL, rS + rL, 2 * rS + rL)}
    pS, pL, pX, pU = pats[rS], pats[rL], pats[rS + rL], pats[2 * rS + rL]
    S, H = O.scatter(pS, Spb), O.scatter(pS, Hpb)
    T = O.hotelling_init(pS, S, pL)
    resid = []
    for _ in range(r["hotelling_steps"]):
        T, res = O.hotelling_step(pS, S, pL, T, pX)
        resid.append(res)
    L0 = O.pm_guess(pS, S, H, pL, T, pX, pL, r["n_electrons"] / 2)
    lnv = O.LNV(pS, S, H, pL, L0, r["n_electrons"], pX, pU)
    start = {"E": lnv.E, "N": lnv.N, "n_corr": lnv.n_corrections_initial}
    steps = []
    for _ in range(r["lnv_steps"]):
        rec = lnv.step()
        steps.append({"E": rec["E"], "N": rec["N"], "gnorm": rec["gnorm"],
                      "n_corr": rec["n_corr"], "restart": bool(rec["restart"]),
                      "fallback": bool(rec["fallback"])})
    eps = sl.eigh(O.to_dense(pS, H), O.to_dense(pS, S), eigvals_only=True)
    n_occ = int(r["n_electrons"]) // 2
    return {"recipe": r,
            "pattern_blocks": {str(R): int(p.nnzb) for R, p in pats.items()},
            "hotelling_residuals": resid, "lnv_start": start, "lnv_steps": steps,
            "dense_band_energy": float(2.0 * eps[:n_occ].sum()),
            "dense_gap": float(eps[n_occ] - eps[n_occ - 1])}


if __name__ == "__main__":
    out = os.path.join(HERE, "si64_reference.json")
    with open(out, "w") as f:
        json.dump(compute(), f, indent=1)
    print("wrote", out)
