"""The whole CUDA pipeline against the stored oracle values of the 64-atom Si cell.

Patterns, Hotelling inversion, Palser-Manolopoulos start and twenty LNV steps run on the
GPU from the raw geometry; the results are compared with tests/golden/si64_reference.json,
written by the oracle alone (no oracle call at test time): exact pattern counts,
residuals to 1e-10 relative, energies and electron counts to 1e-10 Ha/atom, and the same
step decisions.
"""
import json
import os

import pytest
import torch

from paper_2205_08941_gb300 import cq
from paper_2205_08941_gb300 import inputs as I

from helpers import gpu_pattern, upload_pairs

pytestmark = pytest.mark.gpu
REF = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "si64_reference.json")))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_08941_gb300 import build
    build.build()
    c = cq.Context(0)
    yield c
    c.close()


def test_gpu_pipeline_matches_stored_reference(ctx):
    r = REF["recipe"]
    cell = I.diamond_cell(r["ncell"], a=r["a_bohr"], sigma=r["sigma_bohr"], seed=r["seed"],
                          norb=r["norb"])
    Spb, Hpb = I.overlap_hamiltonian(cell, I.silicon_model(r["r_S"]))
    rS, rL = r["r_S"], r["r_L"]
    pats = {R: gpu_pattern(ctx, cell, R) for R in (rS, rL, rS + rL, 2 * rS + rL)}
    for R, p in pats.items():
        assert p.n_blocks == REF["pattern_blocks"][str(R)], R
    pS, pL = pats[rS], pats[rL]
    S, H = upload_pairs(ctx, pS, Spb), upload_pairs(ctx, pS, Hpb)
    T = ctx.zeros(pL)
    ctx.hotelling_init(pS, S, pL, T)
    resid = [ctx.hotelling_step(pS, S, pL, T) for _ in range(r["hotelling_steps"])]
    assert resid == pytest.approx(REF["hotelling_residuals"], rel=1e-10)
    L = ctx.zeros(pL)
    ctx.pm_guess(pS, S, H, pL, T, pL, L, r["n_electrons"] / 2)
    lnv = ctx.lnv(pS, S, H, pL, L, r["n_electrons"])
    tol = 1e-10 * cell.n_atoms
    st = lnv.state()
    assert st["energy"] == pytest.approx(REF["lnv_start"]["E"], abs=tol)
    assert st["n_corr"] == REF["lnv_start"]["n_corr"]
    for k, ref in enumerate(REF["lnv_steps"]):
        rep = lnv.step()
        assert rep["energy"] == pytest.approx(ref["E"], abs=tol), k
        assert rep["n_elec"] == pytest.approx(ref["N"], abs=tol), k
        assert (rep["n_corr"], bool(rep["restart"]), bool(rep["fallback"])) == (
            ref["n_corr"], ref["restart"], ref["fallback"]), k
        assert rep["gnorm"] == pytest.approx(ref["gnorm"], rel=1e-5, abs=1e-9), k
    lnv.close()
