"""The convergence criteria the full-minimisation benchmark reports (CPU, no GPU).

The benchmark times two solvers to the same targets: the energy settled within a tolerance
of the converged FP64 energy (counted on FP64-product energies only, since split-product
energies carry the split's bias), the first FP64 step whose energy change falls below a
tolerance, and the switch out of the split phase when its gradient stops improving.
These tests drive the criteria with synthetic traces and a scripted solver.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_settled_ignores_split_energies_and_waits_for_the_last_excursion():
    e_ref, tol = -100.0, 1e-3
    trace = [(1.0, -100.0, 1e-3, False),      # split energy inside tol: not counted
             (2.0, -99.9, 1e-4, True),         # FP64, outside
             (3.0, -100.0005, 1e-5, True),     # inside ...
             (4.0, -99.99, 1e-6, True),        # ... but leaves again
             (5.0, -100.0002, 1e-7, True),
             (6.0, -99.9999, 1e-8, True)]
    assert bench.settled(trace, e_ref, tol) == 5.0
    assert bench.settled(trace[:2], e_ref, tol) is None


def test_de_stop_compares_consecutive_fp64_energies_only():
    trace = [(1.0, -10.0, 0, False), (2.0, -10.5, 0, True), (3.0, -10.50000001, 0, False),
             (4.0, -10.6, 0, True), (5.0, -10.6000005, 0, True)]
    # the split energy at t=3 sits next to the FP64 one at t=2 but must not stop the run
    assert bench.de_stop(trace, 1e-6) == (5.0, -10.6000005)
    assert bench.de_stop(trace[:4], 1e-6) == (None, None)


class ScriptedLnv:
    """Stands in for the LNV object: each step returns the next scripted RMS gradient."""

    def __init__(self, gnorms):
        self.g = list(gnorms)
        self.k = 0

    def state(self):
        return {"gnorm": self.g[0], "energy": 0.0}

    def step(self):
        self.k += 1
        return {"gnorm": self.g[self.k], "energy": -float(self.k)}


def test_run_until_stops_at_the_gradient_target():
    lnv = ScriptedLnv([1e-2, 5e-3, 1e-3, 5e-4, 1e-4])
    it, st = bench.run_until(lnv, 6e-4, 50)
    assert it == 3 and st["gnorm"] == 5e-4


def test_run_until_leaves_a_stalled_split_phase():
    # falls by 10x per step, then sits at a floor of 1.05e-6 above the 1e-6 target
    g = [1e-3, 1e-4, 1e-5, 1.2e-6, 1.06e-6, 1.05e-6, 1.05e-6, 1.05e-6]
    trace = []
    it, st = bench.run_until(ScriptedLnv(g), 1e-6, 50, trace, 0.0, fp64=False, stall=0.9)
    # step 5 (1.05e-6) still fell by more than 10% against step 3 (1.2e-6); step 6
    # (1.05e-6) did not against step 4 (1.06e-6), so the phase ends there
    assert it == 6 and st["gnorm"] == 1.05e-6
    assert len(trace) == 6 and not any(x[3] for x in trace)
    # without the stall rule the same run only ends at the step cap
    it, _ = bench.run_until(ScriptedLnv(g + [1.05e-6] * 10), 1e-6, 12)
    assert it == 12


@pytest.mark.parametrize("n", [1, 2])
def test_run_until_needs_two_steps_before_judging_a_stall(n):
    g = [1e-3] + [1e-3] * 4
    it, _ = bench.run_until(ScriptedLnv(g), 1e-9, n, stall=0.9)
    assert it == n


class EnergyLnv:
    """Scripted energies with a gradient that never meets its target."""

    def __init__(self, energies):
        self.e = list(energies)
        self.k = 0

    def state(self):
        return {"gnorm": 1.0, "energy": self.e[0]}

    def step(self):
        self.k += 1
        return {"gnorm": 1.0, "energy": self.e[self.k]}


def test_run_until_stops_when_the_energy_settles():
    """The energy-change stop of the default converge leg: the first step whose energy
    differs from the previous one by less than de_tol ends the run."""
    lnv = EnergyLnv([-1.0, -2.0, -2.5, -2.6, -2.6000001, -2.7])
    it, st = bench.run_until(lnv, 1e-8, 50, de_tol=1e-6)
    assert it == 4 and st["energy"] == -2.6000001
    it, _ = bench.run_until(EnergyLnv([-1.0, -2.0, -3.0, -4.0]), 1e-8, 3, de_tol=1e-6)
    assert it == 3  # the step cap still holds


def test_batched_recipe_cells():
    """The 32 cells of the batched workload: seeded (the same cells every call), 500-8000
    atoms each within lattice rounding, densities 0.03-0.06 atoms/A^3, r_L 12-16 bohr,
    species 5/9/13 only."""
    import numpy as np
    a, b = bench.c4_cells(), bench.c4_cells()
    assert len(a) == 32
    for (ca, da, ra), (cb, db, rb) in zip(a, b):
        assert ca.n_atoms == cb.n_atoms and np.array_equal(ca.nb, cb.nb)
        assert np.allclose(ca.pos, cb.pos) and da == db and ra == rb
        assert 500 <= ca.n_atoms <= 8000
        assert 0.03 <= da <= 0.06 and 12.0 <= ra <= 16.0
        assert set(np.unique(ca.nb)) <= {5, 9, 13}
        # the lattice constant realises the drawn density
        vol_a3 = np.prod(ca.box) / 1.8897261254578281 ** 3
        assert ca.n_atoms / vol_a3 == pytest.approx(da, rel=1e-9)
    assert 100000 < sum(c.n_atoms for c, _, _ in a) < 200000


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampled(lines):
    s = bench.ClockSampler(0)
    s.proc = _DoneProcess()
    s.lines = lines
    return s.stop()


def test_clock_samples_give_the_median_and_every_active_reason():
    idle = "Not Active"
    rows = [f"0, {mhz}, 2070, 900.5, 0x0, {idle}, {idle}, {idle}, {cap}"
            for mhz, cap in ((2070, idle), (1980, "Active"), (2070, idle), (2025, idle))]
    rows.insert(1, "0, [N/A], 2070, 0, 0x0, , , , ")   # unreadable sample: skipped
    rows.append("garbage")                               # short line: skipped
    c = _sampled(rows)
    assert c["samples"] == 4
    assert c["sm_mhz"] == 2047.5 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    hot = f"0, 1500, 2070, 1400, 0x48, {idle}, Active, Active, {idle}"
    assert _sampled([hot])["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi_says_so():
    c = bench.ClockSampler(0).stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]
