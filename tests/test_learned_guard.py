"""The guard of the learned start (host logic, no GPU): the learned L is kept only when its
RMS gradient is at most ten times the Palser-Manolopoulos start's and its electron count is
within 1 % of N_e; anything else, NaN included, falls back to the PM start."""
import math

import pytest

from paper_2205_08941_gb300.learned import accept_learned

N_E = 16384.0
PM = {"gnorm": 3.7e-2, "n_elec": N_E}


def state(gnorm, n_elec=N_E):
    return {"gnorm": gnorm, "n_elec": n_elec}


@pytest.mark.parametrize("gnorm,keep", [(2.1e-3, True), (3.7e-1, True), (3.7001e-1, False),
                                        (1.0, False), (0.0, True)])
def test_gradient_ratio(gnorm, keep):
    assert accept_learned(state(gnorm), PM, N_E) is keep


@pytest.mark.parametrize("dn,keep", [(0.0, True), (0.0099 * N_E, True), (-0.0099 * N_E, True),
                                     (0.0101 * N_E, False), (-0.0101 * N_E, False)])
def test_electron_count_within_one_percent(dn, keep):
    assert accept_learned(state(1e-3, N_E + dn), PM, N_E) is keep


def test_nan_and_infinite_states_are_rejected():
    assert not accept_learned(state(math.nan), PM, N_E)
    assert not accept_learned(state(1e-3, math.nan), PM, N_E)
    assert not accept_learned(state(math.inf), PM, N_E)
    assert not accept_learned(state(1e-3), {"gnorm": math.nan, "n_elec": N_E}, N_E)


def test_ratio_is_a_parameter():
    assert accept_learned(state(0.2), PM, N_E, ratio=10.0)
    assert not accept_learned(state(0.2), PM, N_E, ratio=5.0)
