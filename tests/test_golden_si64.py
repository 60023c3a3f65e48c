"""The oracle against its stored reference values for the 64-atom Si cell (CPU).

tests/golden/si64_reference.json was written by tests/golden/make_si64_reference.py from the
oracle and scipy alone.  Recomputing it must give the same pattern counts exactly and the
same residuals, energies and step decisions to rounding, so an accidental change to the
oracle's arithmetic shows up here.  The stored dense-limit band energy bounds the
truncated LNV energy from below.
"""
import json
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_si64_reference as G  # noqa: E402

REF = json.load(open(os.path.join(HERE, "golden", "si64_reference.json")))


@pytest.fixture(scope="module")
def fresh():
    return G.compute()


def test_recipe_is_the_stored_one():
    assert REF["recipe"] == G.RECIPE


def test_pattern_counts_exact(fresh):
    assert fresh["pattern_blocks"] == REF["pattern_blocks"]


def test_hotelling_residuals(fresh):
    assert fresh["hotelling_residuals"] == pytest.approx(REF["hotelling_residuals"], rel=1e-12)
    # quadratic convergence of the residual until the truncation of T stops it
    r = REF["hotelling_residuals"]
    assert r[1] < r[0] and r[2] < r[1]


def test_lnv_start_and_steps(fresh):
    tol = 1e-10 * 64
    assert fresh["lnv_start"]["E"] == pytest.approx(REF["lnv_start"]["E"], abs=tol)
    assert fresh["lnv_start"]["n_corr"] == REF["lnv_start"]["n_corr"]
    for k, (a, b) in enumerate(zip(fresh["lnv_steps"], REF["lnv_steps"])):
        assert a["E"] == pytest.approx(b["E"], abs=tol), k
        assert a["N"] == pytest.approx(b["N"], abs=tol), k
        assert a["gnorm"] == pytest.approx(b["gnorm"], rel=1e-6, abs=1e-12), k
        assert (a["n_corr"], a["restart"], a["fallback"]) == (b["n_corr"], b["restart"],
                                                              b["fallback"]), k


def test_truncated_energy_above_dense_limit():
    # L restricted to a 12-bohr pattern cannot go below the unrestricted minimum 2 sum eps
    assert REF["lnv_steps"][-1]["E"] > REF["dense_band_energy"]
    assert REF["dense_gap"] > 0.1
